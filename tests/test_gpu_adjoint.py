"""GPU adjoint form: far-field adjoint kernel, adjoint solves through torch.autograd,
checked against the oracle's dense gradient and against central finite differences.

Workload: an N = 1024 copy of the parallel-strips scatterer (8 strips 6.4 lambda long,
2 lambda apart, 20 segments per wavelength), leaf 64, eps = 1e-10 (construction floor
~1e-8), 64 observation angles, target t ~ CN(0,1) (seed 1), incidence 30 deg.
Gradient bound vs. the dense oracle: cond(A) * (10 eps_floor + rtol) with eps_floor =
1e-8 and rtol = 1e-10 solves; FD bound 1e-3 relative (solve error / h with h = 1e-4).
"""
import numpy as np
import pytest

import workloads as W
from oracle import efie, farfield

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    from paper_1901_11371_gb300 import autograd as ag
    params = (8.0, 6.4, 2.0)
    g = hb.hb_geometry(W.PARALLEL_STRIPS, params, 1024)
    f = hb.hb_factor(g, 64, 1e-10, form=hb.HB_C128)
    p = efie.Problem(W.PARALLEL_STRIPS, params, 1024)
    a = p.dense(scaled=False)
    phi = W.observation_angles_deg(64)
    t = W.complex_gaussian(64, W.SEED_TARGET)
    return torch, hb, ag, f, p, a, phi, t


def test_far_field_adjoint_matches_dense_transpose(setup):
    torch, hb, ag, f, p, a, phi, t = setup
    gq = W.complex_gaussian(64, 60, 2).T.copy()
    out = hb.hb_far_field_adjoint(f, torch.from_numpy(gq).cuda(), phi).cpu().numpy()
    fm = farfield.far_field_matrix(p, phi)
    for r in range(2):
        ref = fm.conj().T @ gq[r]
        np.testing.assert_allclose(out[r], ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_gradient_vs_dense_oracle(setup):
    torch, hb, ag, f, p, a, phi, t = setup
    b = hb.hb_rhs_plane_wave(f, [30.0]).clone().requires_grad_(True)
    tt = torch.from_numpy(t).cuda()[None, :]
    loss = ag.far_field_loss(f, b, tt, phi, rtol=1e-10, restart=100, maxit=3000)
    loss.backward()
    grad = b.grad.cpu().numpy()[0]
    loss_ref, lam = farfield.loss_gradient(a, p, p.plane_wave(30.0)[:, 0], t, phi)
    bound = np.linalg.cond(a) * (10 * 1e-8 + 1e-10)
    assert abs(loss.item() - loss_ref) <= bound * loss_ref
    assert np.linalg.norm(grad - lam) / np.linalg.norm(lam) <= bound


def test_gradient_vs_central_fd(setup):
    torch, hb, ag, f, p, a, phi, t = setup
    b0 = hb.hb_rhs_plane_wave(f, [30.0])
    tt = torch.from_numpy(t).cuda()[None, :]
    b = b0.clone().requires_grad_(True)
    loss = ag.far_field_loss(f, b, tt, phi, rtol=1e-10, restart=100, maxit=3000)
    loss.backward()
    grad = b.grad.cpu().numpy()[0]
    d = W.complex_gaussian(1024, W.SEED_FD, 32)
    h = 1e-4
    worst = 0.0
    with torch.no_grad():
        for j in range(32):
            dj = torch.from_numpy(d[:, j]).cuda()[None, :]
            lp = ag.far_field_loss(f, b0 + h * dj, tt, phi, rtol=1e-10, restart=100, maxit=3000).item()
            lm = ag.far_field_loss(f, b0 - h * dj, tt, phi, rtol=1e-10, restart=100, maxit=3000).item()
            fd = (lp - lm) / (2 * h)
            an = float(np.real(np.vdot(grad, d[:, j])))
            worst = max(worst, abs(fd - an) / max(abs(fd), 1e-30))
    assert worst <= 1e-3, worst
