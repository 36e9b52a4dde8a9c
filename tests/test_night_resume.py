"""Resumable night runs (paper_1209_5823_gb300.night): host logic on CPU with a stand-in
batch function; the real batch call on the GPU."""
import numpy as np
import pytest

from paper_1209_5823_gb300 import night


class Stop(Exception):
    pass


def _fake(calls):
    def batch(items, precision):
        calls.append([it["id"] for it in items])
        for it in items:
            it["D"] = it["R"] * 2.0
    return batch


def test_resume_skips_recorded_frames(tmp_path):
    ids = [f"f{k:02d}" for k in range(7)]
    out, calls = {}, []
    load = lambda i: {"id": i, "R": np.full(3, float(int(i[1:])))}

    def store_then_stop(i, it):
        out[i] = it["D"].copy()
        if i == "f04":
            raise Stop()

    j = str(tmp_path / "night.journal")
    with pytest.raises(Stop):
        night.run_night(ids, load, store_then_stop, j, group=3, batch=_fake(calls), synchronize=lambda: None)
    # the first group was recorded; the interrupted second one was not
    assert night.read_journal(j) == {"f00", "f01", "f02"}
    done = night.run_night(ids, load, lambda i, it: out.__setitem__(i, it["D"].copy()), j, group=3,
                           batch=_fake(calls), synchronize=lambda: None)
    assert done == ["f03", "f04", "f05", "f06"]
    assert calls == [["f00", "f01", "f02"], ["f03", "f04", "f05"], ["f03", "f04", "f05"], ["f06"]]
    assert night.read_journal(j) == set(ids)
    for i in ids:
        assert np.array_equal(out[i], np.full(3, 2.0 * int(i[1:])))
    # a finished night does nothing
    assert night.run_night(ids, load, lambda i, it: None, j, batch=_fake(calls), synchronize=lambda: None) == []


@pytest.mark.gpu
def test_resumed_night_matches_one_batch(tmp_path):
    import torch
    import paper_1209_5823_gb300 as svk
    import starfield
    specs = starfield.batch_specs(6, scale=0.0625)
    frames = {}
    for s in specs:
        R, I, _ = starfield.frame_pair(s)
        c = starfield.planted_coeffs(49, s.degree, starfield.rng(s.seed + 7)).astype(np.float32)
        frames[s.name] = (torch.from_numpy(R.astype(np.float32)).cuda(), torch.from_numpy(I.astype(np.float32)).cuda(),
                          svk.svk_build_basis(svk.SVK_BASIS_GAUSS, s.L), torch.from_numpy(c).cuda(), s.degree)

    def load(i):
        R, I, B, c, d = frames[i]
        return dict(R=R, I=I, D=torch.empty_like(R), basis=B, coeffs=c, degree=d)

    ref = {i: load(i) for i in frames}
    svk.svk_difference_batch(list(ref.values()))
    torch.cuda.synchronize()
    got = {}
    j = str(tmp_path / "night.journal")

    def store(i, it):
        got[i] = it["D"].clone()
        if len(got) == 3:
            raise Stop()

    with pytest.raises(Stop):
        night.run_night(list(frames), load, store, j, group=2)
    night.run_night(list(frames), load, lambda i, it: got.__setitem__(i, it["D"].clone()), j, group=2)
    for i in frames:
        assert torch.equal(got[i], ref[i]["D"])
