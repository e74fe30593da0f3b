"""Checkpointed adjoint on the GPU against the FP64 oracle's adjoint (which
stores every state), against central finite differences of the GPU forward
in FP64, and through torch.autograd."""
import dataclasses

import numpy as np
import pytest

import oracle
from workloads import Physics, gradient_setup, random_blob_phi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, State, make_params  # noqa: E402
from paper_2304_11165_b300.autograd import adjoint, forward_record, rollout  # noqa: E402


def small_case(seed, ns=2, dims=(21, 17, 13)):
    phi = random_blob_phi(dims, seed, porosity=0.6, ell=1.6)
    phi = np.where(phi > 0, phi * 0.6, phi).astype(np.float32)
    d = (False, True, True, False, False, False)
    phys = Physics(dims=dims, dt=0.06, nspecies=ns, D=(1.0, 0.5), decay=(0.01, 0.2), k_surf=0.7 if ns == 2 else 0.4,
                   dirichlet=d, face_value=(0.0,) * 6)
    rng = np.random.default_rng(seed)
    u0 = rng.uniform(0.2, 1.0, size=(ns,) + phi.shape)
    u0[:, :, :, -1] = 0.0
    u0[:, :, 0, :] = 0.0
    weights = rng.uniform(0, 1, size=(ns,) + phi.shape)
    return phi, phys, u0, weights


def gpu_grad(phi, phys, u0, lamN, nsteps, K, dtype, block=8):
    g = Grid(phi, block=block)
    st = State(g, phys.nspecies, dtype).set_all(u0)
    tape = forward_record(st, make_params(phys), nsteps, K)
    lam = State(g, phys.nspecies, dtype).set_all(lamN)
    grad = adjoint(tape, lam)
    return lam.get_all(), grad, st.get_all(), tape


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("ns,block", [(1, 4), (2, 8), (2, 4)])
def test_fp64_adjoint_equals_oracle_adjoint(ns, block):
    phi, phys, u0, wts = small_case(3 + ns, ns)
    P = oracle.Problem(phi, phys)
    lamN = wts * P.active[None]
    lam0_ref, grad_ref, uN_ref = P.adjoint_run(u0, 30, lamN)
    lam0, grad, uN, _ = gpu_grad(phi, phys, u0, lamN, 30, 7, "f64", block)
    assert rel(uN, uN_ref) < 1e-13
    assert rel(lam0, lam0_ref) < 1e-12
    for s in range(ns):
        assert abs(grad[s] - grad_ref[s]) <= 1e-11 * abs(grad_ref[s]), (s, grad, grad_ref)
    assert abs(grad[2] - grad_ref[ns]) <= 1e-11 * abs(grad_ref[ns])


def test_fp32_adjoint_within_1e4_of_oracle():
    phi, phys, u0, wts = small_case(9, 2)
    P = oracle.Problem(phi, phys)
    lamN = wts * P.active[None]
    lam0_ref, grad_ref, _ = P.adjoint_run(u0, 60, lamN)
    lam0, grad, _, _ = gpu_grad(phi, phys, u0, lamN, 60, 16, "f32", 4)
    assert rel(lam0, lam0_ref) < 1e-4
    for q, qr in ((0, 0), (1, 1), (2, 2)):
        assert abs(grad[q] - grad_ref[qr]) <= 1e-4 * abs(grad_ref[qr])


@pytest.mark.parametrize("block", [4, 8])
@pytest.mark.parametrize("k", [0.0, 0.4])
def test_fp32_one_species_adjoint_within_1e4_of_oracle(block, k):
    """One species (lambda and u^n on the two-row kernel): a box whose block
    count leaves a ragged last group, Dirichlet faces, with and without the
    surface sink; at k = 0 the FP32 path still returns dL/dk, as the FP64 one
    does."""
    phi, phys, u0, wts = small_case(21, 1, dims=(37, 29, 23))
    phys = dataclasses.replace(phys, k_surf=k)
    P = oracle.Problem(phi, phys)
    lamN = wts * P.active[None]
    lam0_ref, grad_ref, _ = P.adjoint_run(u0, 50, lamN)
    lam0, grad, _, _ = gpu_grad(phi, phys, u0, lamN, 50, 8, "f32", block)
    assert rel(lam0, lam0_ref) < 1e-4
    assert abs(grad[0] - grad_ref[0]) <= 1e-4 * abs(grad_ref[0])
    # dL/dk is defined at k = 0 too (the sink's first-order effect)
    assert grad_ref[1] != 0.0
    assert abs(grad[2] - grad_ref[1]) <= 1e-4 * abs(grad_ref[1])


def test_fp64_adjoint_matches_central_differences_of_the_gpu_forward():
    phi, phys, u0, wts = small_case(13, 2)
    nsteps = 40
    _, grad, _, _ = gpu_grad(phi, phys, u0, wts, nsteps, 9, "f64", 8)

    def loss(ph, u_init):
        g = Grid(phi, block=8)
        st = State(g, 2, "f64").set_all(u_init)
        st.step(make_params(ph), nsteps)
        return float((st.get_all() * wts).sum())

    for which, base in (("D0", phys.D[0]), ("D1", phys.D[1]), ("k", phys.k_surf)):
        h = 1e-3 * base

        def at(delta):
            if which == "D0":
                return dataclasses.replace(phys, D=(base + delta, phys.D[1]))
            if which == "D1":
                return dataclasses.replace(phys, D=(phys.D[0], base + delta))
            return dataclasses.replace(phys, k_surf=base + delta)

        fd = (loss(at(h), u0) - loss(at(-h), u0)) / (2 * h)
        g = {"D0": grad[0], "D1": grad[1], "k": grad[2]}[which]
        assert abs(g - fd) <= 1e-6 * abs(fd), (which, g, fd)


def test_autograd_function_gives_the_adjoint_gradients():
    phi, phys, u0, wts = small_case(17, 2)
    g = Grid(phi, block=8)
    c0 = torch.tensor(u0, device="cuda", dtype=torch.float64, requires_grad=True)
    D = torch.tensor(phys.D, dtype=torch.float64, requires_grad=True)
    k = torch.tensor(phys.k_surf, dtype=torch.float64, requires_grad=True)
    w = torch.tensor(wts, device="cuda", dtype=torch.float64)
    uN = rollout(c0, D, k, g, phys, 25, checkpoint_every=6)
    (uN * w).sum().backward()
    lam0, grad, _, _ = gpu_grad(phi, phys, u0, wts, 25, 6, "f64", 8)
    np.testing.assert_allclose(c0.grad.cpu().numpy(), lam0, rtol=0, atol=1e-14 * np.abs(lam0).max())
    np.testing.assert_allclose(D.grad.numpy(), grad[:2], rtol=1e-14)
    assert abs(float(k.grad) - grad[2]) <= 1e-14 * abs(grad[2])
    # direction check of dL/dc0 against central differences of the forward
    v = torch.randn_like(c0) * torch.tensor((oracle.Problem(phi, phys).fixed == 0) *
                                            (oracle.Problem(phi, phys).active > 0), device="cuda")[None]
    h = 1e-4
    with torch.no_grad():
        lp = (rollout(c0 + h * v, D, k, g, phys, 25) * w).sum().item()
        lm = (rollout(c0 - h * v, D, k, g, phys, 25) * w).sum().item()
    fd = (lp - lm) / (2 * h)
    assert abs(float((c0.grad * v).sum()) - fd) <= 1e-7 * abs(fd)


def test_gradient_workload_crop48_against_the_oracle_adjoint():
    """The gradient workload on the 48^3 corner of the 256^3 GRF geometry:
    surface sink k = 0.05, A = 0 held on x = 47, 1000 steps, loss = mean of A
    over pore voxels with x > 42; checkpoints every 64 steps, FP32 state."""
    phi, u0, phys, x_cut = gradient_setup(n=256, crop=48)
    P = oracle.Problem(phi, phys)
    lamN = P.slab_loss_seed(x_cut)
    lam0_ref, grad_ref, uN_ref = P.adjoint_run(u0, phys.steps, lamN)
    lam0, grad, uN, tape = gpu_grad(phi, phys, u0[None], lamN, phys.steps, 64, "f32", 4)
    assert tape.info()["checkpoints"] == 16
    assert rel(uN, uN_ref) < 1e-5
    assert rel(lam0, lam0_ref) < 1e-4
    assert abs(grad[0] - grad_ref[0]) <= 1e-4 * abs(grad_ref[0])
    assert abs(grad[2] - grad_ref[1]) <= 1e-4 * abs(grad_ref[1])
    assert grad_ref[1] < 0  # a stronger surface sink lowers the outlet mean
