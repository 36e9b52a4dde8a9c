"""A night of frames through svk_difference_batch, resumable.

Frames are processed in groups (one batch call each, grouped persistent launches inside);
after a group's results have been handed to the caller, its frame ids are appended to a
journal file (one id per line, flushed and synced).  A run that stops -- an exception in
the caller's code, a killed process -- resumes by calling `run_night` again with the same
journal: frames already recorded there are skipped.
"""
from __future__ import annotations

import os
from typing import Callable, Iterable

from . import SVK_PREC_BF16X3, svk_difference_batch


def read_journal(path: str) -> set[str]:
    if not os.path.exists(path):
        return set()
    with open(path) as f:
        return {line.strip() for line in f if line.strip()}


def _record(path: str, ids: Iterable[str]) -> None:
    with open(path, "a") as f:
        for i in ids:
            f.write(f"{i}\n")
        f.flush()
        os.fsync(f.fileno())


def run_night(frame_ids: Iterable[str], load: Callable[[str], dict], store: Callable[[str, dict], None],
              journal: str, group: int = 8, precision: int = SVK_PREC_BF16X3,
              batch: Callable = svk_difference_batch, synchronize: Callable[[], None] | None = None) -> list[str]:
    """Process every frame id not yet in `journal`; returns the ids processed by this call.

    load(id) -> dict(R, I, D, basis, coeffs, degree) of device tensors (as for
    svk_difference_batch); store(id, item) receives each item once its D is computed (the
    stream is synchronised first).  Ids are recorded in the journal after `store` returned
    for every frame of their group, so a frame is never recorded without its result."""
    if group < 1:
        raise ValueError("group must be >= 1")
    if synchronize is None:
        import torch
        synchronize = torch.cuda.synchronize
    done = read_journal(journal)
    pending = [i for i in frame_ids if i not in done]
    processed = []
    for s in range(0, len(pending), group):
        ids = pending[s:s + group]
        items = [load(i) for i in ids]
        batch(items, precision=precision)
        synchronize()
        for i, it in zip(ids, items):
            store(i, it)
        _record(journal, ids)
        processed.extend(ids)
    return processed
