"""GPU parity of the adjoint gradient against the FP64 oracle (state-vector adjoint and
central finite differences of the elimination oracle, h = 1e-4)."""
import numpy as np
import pytest

import circuitgen as cg
from oracle import statevector as SV
from oracle import ve as VE

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
q = pytest.importorskip("paper_1805_01450_gb300")


def tol(n):
    return 1e-5 * 2.0 ** (-n / 2)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("kw", [dict(), dict(n_slices=3, inner_slices=1), dict(n_slices=4, inner_slices=2,
                                                                                host_merge_rank=0)])
def test_rotation_3x4_all_angles_vs_adjoint_oracle(kw):
    c = cg.rotation_circuit(3, 4, 8, 41)
    p = q.Plan(c, gradient=True, **kw)
    xs = cg.random_bitstrings(12, 3, 42)
    a, g = p.amplitude_grad(xs)
    a, g = a.cpu().numpy(), g.cpu().numpy()
    assert g.shape == (3, c.n_params)
    for i, x in enumerate(xs):
        a_ref, g_ref = SV.sv_adjoint_grad(c, x)
        assert abs(a[i] - a_ref) < tol(12)
        assert np.max(np.abs(g[i] - g_ref)) < tol(12)


def test_gradient_checkpointing_on_device():
    # a memory budget of half one work item's gradient arena: forward values are recomputed in
    # the backward pass; gradients as the state-vector adjoint and as the plan that keeps all
    c = cg.rotation_circuit(4, 4, 16, 9)
    full = q.Plan(c, gradient=True, n_slices=0)
    small = q.Plan(c, gradient=True, n_slices=0, order=full.order,
                   mem_budget_bytes=full.info["grad_arena_bytes"] // 2)
    assert small.info["grad_recomputed"] > 0
    xs = cg.random_bitstrings(16, 3, 11)
    a, g = (t.cpu().numpy() for t in small.amplitude_grad(xs))
    a_full, g_full = (t.cpu().numpy() for t in full.amplitude_grad(xs))
    assert np.max(np.abs(g - g_full)) < tol(16) and np.max(np.abs(a - a_full)) < tol(16)
    for i, x in enumerate(xs):
        a_ref, g_ref = SV.sv_adjoint_grad(c, x)
        assert abs(a[i] - a_ref) < tol(16)
        assert np.max(np.abs(g[i] - g_ref)) < tol(16)


def test_thetas_override_and_repeat():
    c = cg.rotation_circuit(3, 3, 6, 43)
    p = q.Plan(c, gradient=True, n_slices=2)
    x = 0b101010101
    rng = np.random.default_rng(1)
    ws = p.workspace(1)
    for _ in range(2):
        th = rng.uniform(0, 2 * np.pi, c.n_params)
        a, g = p.amplitude_grad([x], torch.tensor(th, device="cuda"), workspace=ws)
        a_ref, g_ref = SV.sv_adjoint_grad(SV.with_thetas(c, th), x)
        assert abs(a.cpu().numpy()[0] - a_ref) < tol(9)
        assert np.max(np.abs(g.cpu().numpy()[0] - g_ref)) < tol(9)
    # the workspace now holds the last angles: amplitude() agrees with the oracle at them
    assert abs(p.amplitude([x], workspace=ws).cpu().numpy()[0] - a_ref) < tol(9)


def test_5x5x20_rotation_circuit_finite_differences():
    # 1000 angles; central differences of the elimination oracle on a seeded 64 of them
    c = cg.rotation_circuit(5, 5, 20, 4001)
    p = q.Plan(c, gradient=True, n_slices=6)
    x = cg.random_bitstrings(25, 1, 4002)[0]
    a, g = p.amplitude_grad([x])
    a, g = a.cpu().numpy()[0], g.cpu().numpy()[0]
    assert g.shape == (1000,)
    order = q.Plan(c, n_slices=0, host_merge_rank=0).order
    assert abs(a - VE.ve_amplitude(c, x, order)) < tol(25)
    th = np.array(c.thetas())
    h = 1e-4
    for pi in np.random.default_rng(4003).choice(1000, 64, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[pi] += h
        tm[pi] -= h
        fd = (VE.ve_amplitude(SV.with_thetas(c, tp), x, order) -
              VE.ve_amplitude(SV.with_thetas(c, tm), x, order)) / (2 * h)
        assert abs(g[pi] - fd) < tol(25), pi


def test_shared_memory_and_global_gradient_kernels_agree():
    # 5x5x20 rotation circuit, all 1000 angles: 1 sliced variable leaves the gradient arena
    # too large for shared memory (global-memory kernel); 8 let it fit (on-chip kernel; 512
    # work items for two bitstrings, more than one staged CTA per SM could take at once);
    # 6 give 128 work items, each with a CTA of the staged form (leaf data on chip too)
    c = cg.rotation_circuit(5, 5, 20, 4001)
    xs = cg.random_bitstrings(25, 2, 4004)
    big = q.Plan(c, gradient=True, n_slices=1, inner_slices=0)
    small = q.Plan(c, gradient=True, n_slices=8, inner_slices=0)
    staged = q.Plan(c, gradient=True, n_slices=6, inner_slices=0)
    assert big.info["grad_smem_bytes"] > 232448 and 0 < small.info["grad_smem_bytes"] <= 232448
    a1, g1 = (t.cpu().numpy() for t in big.amplitude_grad(xs))
    a2, g2 = (t.cpu().numpy() for t in small.amplitude_grad(xs))
    a3, g3 = (t.cpu().numpy() for t in staged.amplitude_grad(xs))
    assert np.max(np.abs(a1 - a2)) < tol(25) and np.max(np.abs(g1 - g2)) < tol(25)
    assert np.max(np.abs(a3 - a2)) < tol(25) and np.max(np.abs(g3 - g2)) < tol(25)
    order = q.Plan(c, n_slices=0, host_merge_rank=0).order
    for i, x in enumerate(xs):
        assert abs(a2[i] - VE.ve_amplitude(c, x, order)) < tol(25)


def test_autograd_function_norm_squared():
    from paper_1805_01450_gb300.autograd import amplitude
    c = cg.rotation_circuit(2, 3, 5, 44)
    p = q.Plan(c, gradient=True)
    xs = [0b000111, 0b101010]
    th = torch.tensor(c.thetas(), dtype=torch.float64, device="cuda", requires_grad=True)
    a = amplitude(p, xs, th)
    loss = (a.abs() ** 2).sum()
    (gt,) = torch.autograd.grad(loss, th)
    want = np.zeros(c.n_params)
    for x in xs:
        a_ref, g_ref = SV.sv_adjoint_grad(c, x)
        want += 2 * np.real(np.conj(a_ref) * g_ref)
    assert np.max(np.abs(gt.cpu().numpy() - want)) < 1e-5


def test_gradient_errors():
    c = cg.rotation_circuit(2, 2, 2, 45)
    p = q.Plan(c)                                # no gradient program
    with pytest.raises(q.QvxError):
        p.amplitude_grad([0])
    pg = q.Plan(c, gradient=True)
    with pytest.raises(q.QvxError):
        pg.amplitude_grad([0], torch.zeros(3, dtype=torch.float64))
