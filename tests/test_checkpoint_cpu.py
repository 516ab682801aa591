"""Checkpoint and resume of an amplitude over its slice ranges (host logic; the GPU call is
replaced by a host stand-in that computes each range's partial sums with the oracle)."""
import json

import numpy as np
import pytest

import circuitgen as cg
from oracle import statevector as SV
from oracle import ve as VE

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")
from paper_1805_01450_gb300.checkpoint import amplitude_resumable  # noqa: E402


class _StandIn:
    """The plan calls amplitude_resumable makes, answered on the host: image(),
    n_slice_terms and amplitude(bitstrings, slice_begin, slice_count)."""

    def __init__(self, circ, n_slices):
        self.circ = circ
        self.plan = q.Plan(circ, n_slices=n_slices)
        self.n_slice_terms = self.plan.n_slice_terms
        self.calls = []

    def image(self):
        return self.plan.image()

    def amplitude(self, bitstrings, slice_begin=0, slice_count=None):
        self.calls.append((slice_begin, slice_count))
        ids = np.arange(slice_begin, slice_begin + slice_count, dtype=np.int64)
        return torch.tensor([VE.exact_sum(VE.slice_terms(self.circ, x, self.plan.order, self.plan.slices,
                                                         slice_ids=ids)) for x in bitstrings],
                            dtype=torch.complex128)


def test_interrupted_run_resumes_to_the_same_amplitudes(tmp_path):
    circ = cg.grid_circuit(4, 4, 12, 7)
    xs = cg.random_bitstrings(16, 3, 8)
    want = SV.final_state(circ)[xs]
    path = str(tmp_path / "journal.jsonl")
    p = _StandIn(circ, 5)                                   # 32 slice terms, 7 ranges of 5
    assert amplitude_resumable(p, xs, path, 5, stop_after=3) is None
    assert len(p.calls) == 3
    p2 = _StandIn(circ, 5)
    got = amplitude_resumable(p2, xs, path, 5)
    assert [c[0] for c in p2.calls] == [15, 20, 25, 30]    # only the missing ranges
    assert np.max(np.abs(got - want)) < 1e-14
    p3 = _StandIn(circ, 5)
    assert np.array_equal(amplitude_resumable(p3, xs, path, 5), got) and p3.calls == []
    full = amplitude_resumable(_StandIn(circ, 5), xs, str(tmp_path / "other.jsonl"), 5)
    assert np.array_equal(full, got)


def test_cut_line_is_recomputed_and_foreign_journal_refused(tmp_path):
    circ = cg.grid_circuit(4, 4, 12, 7)
    xs = cg.random_bitstrings(16, 2, 9)
    path = tmp_path / "journal.jsonl"
    p = _StandIn(circ, 4)
    amplitude_resumable(p, xs, str(path), 4, stop_after=2)
    lines = path.read_text().splitlines()
    path.write_text("\n".join(lines[:-1] + [lines[-1][:20]]) + "\n")   # the last line cut short
    p2 = _StandIn(circ, 4)
    got = amplitude_resumable(p2, xs, str(path), 4)
    assert p2.calls[0] == (4, 4)
    assert np.max(np.abs(got - SV.final_state(circ)[xs])) < 1e-14
    other = cg.random_bitstrings(16, 2, 10)
    with pytest.raises(ValueError):
        amplitude_resumable(_StandIn(circ, 4), other, str(path), 4)
    head = json.loads(path.read_text().splitlines()[0])
    assert head["slice_terms"] == 16 and head["range_slices"] == 4


def test_records_after_a_cut_line_are_kept(tmp_path):
    circ = cg.grid_circuit(4, 4, 12, 7)
    xs = cg.random_bitstrings(16, 2, 9)
    path = tmp_path / "journal.jsonl"
    amplitude_resumable(_StandIn(circ, 4), xs, str(path), 4, stop_after=1)
    with open(path, "a") as f:
        f.write('{"begin": 4, "co')                        # an append cut short
    amplitude_resumable(_StandIn(circ, 4), xs, str(path), 4, stop_after=2)   # ranges 4 and 8
    p = _StandIn(circ, 4)
    got = amplitude_resumable(p, xs, str(path), 4)
    assert p.calls == [(12, 4)]
    assert np.max(np.abs(got - SV.final_state(circ)[xs])) < 1e-14
