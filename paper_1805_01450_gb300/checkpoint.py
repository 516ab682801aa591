"""Checkpoint and resume of one amplitude computation over its slice ranges.

The 2^k slice terms of an amplitude are independent (Section 3.B.2), so a long computation
(many sliced variables, or a 9 x 9 grid) can be split into ranges that are computed one by
one and recorded as they finish. The journal is a text file of JSON lines: a header naming
the plan (a hash of its device image, which fixes the circuit, order, slices and program)
and the bitstrings, then one line per finished range with its FP64 partial sums. A run that
stops (a crash, a preempted job) resumes by reading the journal, skipping the ranges it
records and computing the rest; the amplitudes are the ranges' partials added in range
order with compensation, so a resumed run gives the same result as an uninterrupted one.
A journal written for another plan or other bitstrings is refused, not reused.
"""
from __future__ import annotations

import hashlib
import json
import os

from .distributed import compensated_sum


def plan_key(plan, bitstrings) -> str:
    """Hash of the plan's device image and the bitstrings: what a journal belongs to."""
    h = hashlib.sha256()
    h.update(plan.image())
    h.update(json.dumps([int(b) for b in bitstrings]).encode())
    return h.hexdigest()


def _read(path, key):
    done = {}
    if not os.path.exists(path):
        return done
    with open(path) as f:
        lines = [l for l in f.read().splitlines() if l.strip()]
    if not lines:
        return done
    head = json.loads(lines[0])
    if head.get("key") != key:
        raise ValueError(f"{path}: journal of another plan or other bitstrings")
    for l in lines[1:]:
        try:
            r = json.loads(l)
        except json.JSONDecodeError:   # a line cut short by an interruption: recomputed
            continue
        done[(r["begin"], r["count"])] = [complex(re, im) for re, im in r["partial"]]
    return done


def amplitude_resumable(plan, bitstrings, path, range_slices, stop_after=None):
    """The amplitudes of `bitstrings` (complex128 numpy array) computed over slice ranges of
    `range_slices` terms, journalled to `path`. `stop_after` ends the call after that many
    newly computed ranges and returns None (what an interrupted run leaves behind)."""
    import numpy as np
    total = plan.n_slice_terms
    if range_slices < 1:
        raise ValueError("range_slices must be positive")
    key = plan_key(plan, bitstrings)
    done = _read(path, key)
    if not os.path.exists(path) or os.path.getsize(path) == 0:
        with open(path, "w") as f:
            f.write(json.dumps({"key": key, "slice_terms": total, "range_slices": range_slices}) + "\n")
    else:
        with open(path, "rb") as f:
            f.seek(-1, os.SEEK_END)
            cut = f.read(1) != b"\n"
        if cut:   # end the cut line, so that the next record starts a line of its own
            with open(path, "a") as f:
                f.write("\n")
    ranges = [(b, min(range_slices, total - b)) for b in range(0, total, range_slices)]
    fresh = 0
    for b, n in ranges:
        if (b, n) in done:
            continue
        if stop_after is not None and fresh >= stop_after:
            return None
        part = plan.amplitude(bitstrings, slice_begin=b, slice_count=n).cpu().numpy()
        done[(b, n)] = [complex(v) for v in part]
        with open(path, "a") as f:
            f.write(json.dumps({"begin": b, "count": n,
                                "partial": [[v.real, v.imag] for v in done[(b, n)]]}) + "\n")
            f.flush()
            os.fsync(f.fileno())
        fresh += 1
    parts = np.array([done[r] for r in ranges], dtype=np.complex128)
    return compensated_sum(parts)
