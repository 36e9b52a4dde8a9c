"""Tensor-core plans whose basis slices stream through a shared-memory ring (large kernels,
where resident tables leave room only for narrow blocks): parity with the FP64 oracle,
agreement to FP32 rounding with the resident-table plan of the same block height, row
bands, batches of frames with distinct bases, the four-lane epilogue at 49..56 stamps, and
the plan rules of svk_set_plan.  Also the FP16x2 precision (an FP16-exact basis, two MMAs
per K step) on resident and streamed plans."""
import numpy as np
import pytest
import torch

import paper_1209_5823_gb300 as svk
from _helpers import TOL_FP32, coeffs, oracle_conv, rel_err, star_pair

pytestmark = pytest.mark.gpu

SPLIT = [svk.SVK_PREC_BF16X3, svk.SVK_PREC_FP16X3]


@pytest.fixture(autouse=True)
def _default_plans():
    """Plans are per process: every test leaves the defaults behind."""
    yield
    for L in range(1, 32, 2):
        for p in (svk.SVK_PREC_BF16X3, svk.SVK_PREC_FP16X3, svk.SVK_PREC_BF16, svk.SVK_PREC_FP16X2):
            svk.svk_set_plan(49, L, p, 0)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _frame(W, H, L, d, seed):
    R, I = star_pair(W, H, max(3, W * H // 300), 700 + seed + W + H)
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    c = coeffs(49, d, 31 + seed)
    return R, I, B, c


def _conv(R, B, c, d, prec):
    out = svk.svk_convolve(_dev(R), B, _dev(c), d, method=svk.SVK_METHOD_BASIS, precision=prec)
    torch.cuda.synchronize()
    return out


def test_default_plan_streams_only_large_kernels():
    for L, streamed in ((11, 0), (19, 0), (23, 0), (25, 1), (31, 1)):
        G, stages, sm = svk.svk_tc_plan(49, L, svk.SVK_PREC_BF16X3)
        assert sm == streamed, L
        assert G == 5  # 245 of 256 MMA columns at every kernel size
        if sm:
            assert stages == 16
    # the T-factored form's few stamps keep resident tables and tall blocks
    G, _, sm = svk.svk_tc_plan(6, 31, svk.SVK_PREC_BF16X3)
    assert sm == 0 and G > 5


@pytest.mark.parametrize("L,G,prec", [
    (31, 1, svk.SVK_PREC_BF16X3),   # the one block height resident tables allow at L = 31
    (27, 2, svk.SVK_PREC_FP16X3),
    (25, 3, svk.SVK_PREC_BF16X3),
    (21, 4, svk.SVK_PREC_BF16X3),   # odd tap-group count: paired last groups, zero partner tile
    (17, 4, svk.SVK_PREC_FP16X3),
    (25, 5, svk.SVK_PREC_BF16),     # one part: resident G = 5 fits too
])
def test_streamed_equals_resident(L, G, prec):
    W, H, d = 300, 53, 2
    R, _, B, c = _frame(W, H, L, d, L + G)
    res = {}
    for sm in (0, 1):
        stages = [16, 8, 4] if sm == 0 else [16]
        for st in stages:
            try:
                svk.svk_set_plan(49, L, prec, G, st, sm)
                break
            except svk.SvkError:
                continue
        else:
            pytest.fail(f"no plan G={G} streamed={sm} for L={L}")
        assert svk.svk_tc_plan(49, L, prec)[0::2] == (G, sm)
        res[sm] = _conv(R, B, c, d, prec)
    # the same MMAs on the same operands in the same order; the streamed kernel's epilogue
    # sums the 49 stamps in four-lane groups, the resident one per lane, so the two agree to
    # FP32 rounding (a slice read from the wrong slot would differ at the 1e-2 level)
    scale = res[0].abs().max().item()
    assert (res[1] - res[0]).abs().max().item() <= 2.0 ** -20 * scale
    if prec != svk.SVK_PREC_BF16:
        ref = oracle_conv(R, B.cpu().numpy(), c, d)
        assert rel_err(res[1].cpu().numpy(), ref) <= TOL_FP32


@pytest.mark.parametrize("prec", SPLIT)
@pytest.mark.parametrize("W,H,L,d", [
    (260, 40, 25, 3),
    (129, 37, 27, 1),
    (300, 23, 29, 2),
    (130, 23, 31, 2),
    (1000, 3, 31, 0),    # fewer rows than a block: one block band, most slices beyond the frame
    (5, 61, 31, 2),      # L > W
    (1, 1, 25, 2),       # 1x1 frame
])
def test_streamed_default_matches_oracle(W, H, L, d, prec):
    assert svk.svk_tc_plan(49, L, prec)[2] == 1
    R, I, B, c = _frame(W, H, L, d, 3)
    D = svk.svk_difference(_dev(R), _dev(I), B, _dev(c), d, method=svk.SVK_METHOD_BASIS, precision=prec)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    assert rel_err(D.cpu().numpy() + I, ref) <= TOL_FP32


@pytest.mark.parametrize("G", [5, 3, 1])
def test_streamed_block_heights_agree(G):
    # an even tap-group count (L = 29: 4 groups): no pairing, so the tensor cores accumulate
    # every pixel's C_k in the same order whatever the block height (only exact zeros are
    # added); the epilogue splits the stamps over lanes by the row's accumulator column
    # modulo 8, which follows the block height, so the results agree to FP32 rounding
    L, d, prec = 29, 2, svk.SVK_PREC_BF16X3
    R, _, B, c = _frame(200, 47, L, d, 9)
    base = _conv(R, B, c, d, prec)  # default: streamed, G = 5
    svk.svk_set_plan(49, L, prec, G, 16, 1)
    other = _conv(R, B, c, d, prec)
    scale = base.abs().max().item()
    assert (other - base).abs().max().item() <= 2.0 ** -20 * scale


@pytest.mark.parametrize("prec", SPLIT)
@pytest.mark.parametrize("N,L,d", [
    # the streamed kernel's epilogue reads each output row's columns from the 8-column
    # boundary below its first one, in 7 or 8 repetitions of 8 columns
    (50, 9, 2),    # 5-row blocks; the first row's window ends at the MMA's last column
    (52, 11, 3),   # 4-row blocks, rows starting 4 columns past a boundary
    (53, 13, 1),   # 4-row blocks, 8 repetitions for rows starting 5 or 7 columns past one
    (56, 9, 3),    # 4-row blocks, every row on a boundary
])
def test_streamed_stamp_counts_50_to_56(N, L, d, prec):
    W, H = 230, 47
    R, I = star_pair(W, H, max(3, W * H // 300), 600 + N)
    B = svk.svk_build_basis(svk.SVK_BASIS_DELTA, L)[:N].contiguous()
    c = coeffs(N, d, N)
    svk.svk_set_plan(N, L, prec, 256 // N, 16, 1)
    try:
        assert svk.svk_tc_plan(N, L, prec) == (256 // N, 16, 1)
        D = svk.svk_difference(_dev(R), _dev(I), B, _dev(c), d, method=svk.SVK_METHOD_BASIS, precision=prec)
    finally:
        svk.svk_set_plan(N, L, prec, 0)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    assert rel_err(D.cpu().numpy() + I, ref) <= TOL_FP32


def test_streamed_row_bands():
    L, d, prec = 31, 2, svk.SVK_PREC_BF16X3
    W, H = 257, 90
    R, I, B, c = _frame(W, H, L, d, 5)
    Rt, It, ct = _dev(R), _dev(I), _dev(c)
    whole = svk.svk_difference(Rt, It, B, ct, d, method=svk.SVK_METHOD_BASIS, precision=prec)
    gran = svk.svk_band_rows(svk.SVK_METHOD_BASIS, prec, 49, L, d)
    assert gran == 5
    cuts = [0, 4 * gran, 11 * gran, H]
    for y0, ye in zip(cuts[:-1], cuts[1:]):
        r0, r1 = max(0, y0 - L // 2), min(H, ye + L // 2)
        Db = svk.svk_difference_rows(Rt[r0:r1].contiguous(), It[y0:ye].contiguous(), B, ct, d, W, H, y0, ye, r0,
                                     method=svk.SVK_METHOD_BASIS, precision=prec)
        assert torch.equal(Db, whole[y0:ye]), (y0, ye)


def test_streamed_batch_with_distinct_bases():
    # frames of one (N, L) share a launch; each streams its own basis's slices, so frames
    # with different bases need no reload between them
    L, prec = 27, svk.SVK_PREC_BF16X3
    Bg = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L)
    Bs = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, L, sigma=(0.9, 1.8, 3.0))
    items = []
    for k, (W, H, d, B) in enumerate(((300, 70, 2, Bg), (129, 41, 3, Bs), (260, 33, 1, Bg), (77, 90, 0, Bs))):
        R, I = star_pair(W, H, max(3, W * H // 300), 900 + k)
        items.append(dict(R=_dev(R), I=_dev(I), D=torch.empty((H, W), device="cuda"), basis=B,
                          coeffs=_dev(coeffs(49, d, 80 + k)), degree=d))
    svk.svk_difference_batch(items, precision=prec)
    torch.cuda.synchronize()
    for it in items:
        one = svk.svk_difference(it["R"], it["I"], it["basis"], it["coeffs"], it["degree"],
                                 method=svk.SVK_METHOD_BASIS, precision=prec)
        assert torch.equal(one, it["D"])
    it = items[1]
    ref = oracle_conv(it["R"].cpu().numpy(), Bs.cpu().numpy(), it["coeffs"].cpu().numpy(), 3)
    assert rel_err(it["D"].cpu().numpy() + it["I"].cpu().numpy(), ref) <= TOL_FP32


def test_set_plan_rules():
    p = svk.SVK_PREC_BF16X3
    with pytest.raises(svk.SvkError):
        svk.svk_set_plan(49, 31, p, 5, 4, 1)    # a streamed ring needs 8 or 16 stages
    with pytest.raises(svk.SvkError):
        svk.svk_set_plan(49, 21, p, 5, 16, 1)   # odd tap groups: G - 1 + 1 > 16 / 4
    with pytest.raises(svk.SvkError):
        svk.svk_set_plan(49, 31, p, 5, 16, 0)   # resident tables do not fit
    with pytest.raises(svk.SvkError):
        svk.svk_set_plan(49, 31, p, 6, 16, 1)   # 294 MMA columns
    svk.svk_set_plan(49, 31, p, 2, 8, 1)
    assert svk.svk_tc_plan(49, 31, p) == (2, 8, 1)
    assert svk.svk_band_rows(svk.SVK_METHOD_BASIS, p, 49, 31, 2) == 2
    svk.svk_set_plan(49, 31, p, 0)
    assert svk.svk_tc_plan(49, 31, p) == (5, 16, 1)


# ---------------------------------------------------------------- FP16x2 (FP16-exact basis)

def test_round_basis_fp16_is_exact_and_idempotent():
    B = svk.svk_build_basis(svk.SVK_BASIS_GAUSS, 19)
    Br = svk.svk_round_basis_fp16(B.clone())
    v = Br.cpu().numpy().astype(np.float64) * 1024.0
    assert np.array_equal(v.astype(np.float16).astype(np.float64), v)  # 1024 b is an FP16 value
    assert np.abs(Br.cpu().numpy() - B.cpu().numpy()).max() <= 2.0 ** -11 * np.abs(B.cpu().numpy()).max()
    assert torch.equal(svk.svk_round_basis_fp16(Br.clone()), Br)


@pytest.mark.parametrize("W,H,L,d", [
    (300, 77, 19, 2),    # paired last tap groups (3 groups)
    (260, 40, 25, 3),    # streamed slices
    (130, 23, 31, 2),
    (129, 37, 15, 1),
    (47, 38, 7, 3),
    (1, 1, 11, 2),
])
def test_fp16x2_matches_oracle_on_a_rounded_basis(W, H, L, d):
    R, I, B, c = _frame(W, H, L, d, 17)
    B = svk.svk_round_basis_fp16(B)
    D = svk.svk_difference(_dev(R), _dev(I), B, _dev(c), d, method=svk.SVK_METHOD_BASIS,
                           precision=svk.SVK_PREC_FP16X2)
    ref = oracle_conv(R, B.cpu().numpy(), c, d)
    assert rel_err(D.cpu().numpy() + I, ref) <= TOL_FP32


@pytest.mark.parametrize("L,G", [(31, 5), (25, 5), (21, 4)])
def test_fp16x2_streamed_equals_resident(L, G):
    p = svk.SVK_PREC_FP16X2
    R, _, B, c = _frame(220, 41, L, 2, 23)
    B = svk.svk_round_basis_fp16(B)
    res = {}
    for sm, stages in ((1, [16]), (0, [16, 8, 4])):
        for st in stages:
            try:
                svk.svk_set_plan(49, L, p, G, st, sm)
                break
            except svk.SvkError:
                continue
        else:
            continue  # no resident plan of this height: the streamed one alone is checked below
        res[sm] = _conv(R, B, c, 2, p)
    if 0 in res:  # equal to FP32 rounding (the two epilogues sum the stamps in different orders)
        assert (res[1] - res[0]).abs().max().item() <= 2.0 ** -20 * res[0].abs().max().item()
    ref = oracle_conv(R, B.cpu().numpy(), c, 2)
    assert rel_err(res[1].cpu().numpy(), ref) <= TOL_FP32


def test_fp16x2_is_the_basis_form_only():
    R, _, B, c = _frame(64, 32, 11, 1, 29)
    with pytest.raises(svk.SvkError):
        svk.svk_convolve(_dev(R), B, _dev(c), 1, method=svk.SVK_METHOD_TFORM, precision=svk.SVK_PREC_FP16X2)
    with pytest.raises(svk.SvkError):
        svk.svk_convolve(_dev(R), B, _dev(c), 1, method=svk.SVK_METHOD_DIRECT, precision=svk.SVK_PREC_FP16X2)
