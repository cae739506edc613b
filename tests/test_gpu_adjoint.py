"""GPU adjoint: gradients of J(u0, beta) from the hand-written CUDA reverse
sweep against (1) the oracle's reverse sweep, whose local derivatives are
complex steps of the oracle's own collision, (2) central finite differences
of the GPU forward map in FP64, (3) itself under different checkpoint
intervals, and (4) the FP32 adjoint against the FP64 one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_1507_02509_gb300 import Lattice, capi, flows  # noqa: E402
from paper_1507_02509_gb300.autograd import kbc_objective  # noqa: E402

pytestmark = pytest.mark.gpu

OV = {"lbgk": O.LBGK, "A": O.A, "B": O.B, "C": O.C, "D": O.D}


def _case(n, seed, k0=2.0, urms=0.05):
    rho, ux, uy = flows.turbulence(n, k0=k0, urms=urms, seed=seed, kcut=max(2, n // 4))
    rng = np.random.default_rng(seed + 1)
    rho = rho + 0.01 * rng.standard_normal(rho.shape)
    tx = 0.03 * rng.standard_normal((n, n))
    ty = 0.03 * rng.standard_normal((n, n))
    return rho, ux, uy, tx, ty


def _gpu_adjoint(variant, dtype, beta, rho, ux, uy, steps, K, objective, tx=None, ty=None,
                 guard=None, gamma=None):
    ny, nx = rho.shape
    lat = Lattice(nx, ny, variant=variant, beta=beta, dtype=dtype)
    if guard is not None:
        lat.set_guard(guard)
    if gamma is not None:
        lat.set_gamma(gamma)
    u = np.ascontiguousarray(np.stack((ux, uy)))
    tgt = np.ascontiguousarray(np.stack((tx, ty))) if objective == 1 else None
    g = np.empty((2, ny, nx))
    J, gb = capi.kbc_adjoint(lat.h, np.ascontiguousarray(rho), u, steps, K, objective, tgt, g)
    lat.close()
    return J, g, gb


@pytest.mark.parametrize("objective", [0, 1])
@pytest.mark.parametrize("variant", ["lbgk", "A", "B", "C", "D"])
def test_adjoint_matches_oracle_adjoint(variant, objective):
    """16x16, 12 steps, FP64: J to 1e-13 and gradients to 1e-9 (relative, in
    the max norm) against the oracle's complex-step reverse sweep."""
    n, steps, beta = 16, 12, 0.95
    rho, ux, uy, tx, ty = _case(n, 5)
    J, g, gb = _gpu_adjoint(variant, "f64", beta, rho, ux, uy, steps, 5, objective, tx, ty)
    Jo, gxo, gyo, gbo = O.adjoint(OV[variant], beta, rho, ux, uy, steps, objective, tx, ty)
    assert J == pytest.approx(Jo, rel=1e-13)
    go = np.stack((gxo, gyo))
    assert np.max(np.abs(g - go)) <= 1e-9 * np.max(np.abs(go))
    assert gb == pytest.approx(gbo, rel=1e-9)


@pytest.mark.parametrize("objective", [0, 1])
@pytest.mark.parametrize("variant", ["A", "B", "C", "D"])
def test_fixed_gamma_adjoint_matches_oracle_adjoint(variant, objective):
    """Regularised mode, gamma fixed at 1/beta (the regularised limit of
    Sec. 4): the reverse sweep's fixed-gamma branch, including its beta
    derivative through beta (gamma - 2), against the oracle's complex-step
    sweep in the same mode (16x16, 12 steps, FP64: J to 1e-13, gradients to
    1e-9)."""
    n, steps, beta = 16, 12, 0.95
    rho, ux, uy, tx, ty = _case(n, 7)
    J, g, gb = _gpu_adjoint(variant, "f64", beta, rho, ux, uy, steps, 5, objective, tx, ty,
                            gamma=1.0 / beta)
    Jo, gxo, gyo, gbo = O.adjoint(OV[variant], beta, rho, ux, uy, steps, objective, tx, ty,
                                  gamma_mode=1, gamma_fixed=1.0 / beta)
    assert J == pytest.approx(Jo, rel=1e-13)
    go = np.stack((gxo, gyo))
    assert np.max(np.abs(g - go)) <= 1e-9 * np.max(np.abs(go))
    assert gb == pytest.approx(gbo, rel=1e-9)


@pytest.mark.parametrize("variant", ["B", "C"])
def test_adjoint_matches_finite_differences(variant):
    """64x64 (vector-row kernel), 40 steps, FP64: dJ/du0 at three nodes and
    dJ/dbeta against central differences of the GPU forward map (h = 1e-6
    relative agreement 1e-6)."""
    n, steps, beta = 64, 40, 0.97
    rho, ux, uy, tx, ty = _case(n, 8, k0=3.0, urms=0.04)
    J, g, gb = _gpu_adjoint(variant, "f64", beta, rho, ux, uy, steps, 10, 1, tx, ty)

    def J_of(ux_, uy_, b):
        lat = Lattice(n, n, variant=variant, beta=b, dtype="f64")
        lat.init(rho, ux_, uy_).step(steps)
        _, vx, vy = (t.cpu().numpy() for t in lat.moments())
        lat.close()
        return 0.5 * np.sum((vx - tx) ** 2 + (vy - ty) ** 2)

    assert J == pytest.approx(J_of(ux, uy, beta), rel=1e-12)
    h = 1e-6
    for (yy, xx) in ((3, 5), (40, 17), (63, 63)):
        for comp in (0, 1):
            up, um = (ux.copy(), uy.copy()), (ux.copy(), uy.copy())
            up[comp][yy, xx] += h
            um[comp][yy, xx] -= h
            fd = (J_of(*up, beta) - J_of(*um, beta)) / (2 * h)
            assert g[comp, yy, xx] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(J)), (yy, xx, comp)
    fd = (J_of(ux, uy, beta + h) - J_of(ux, uy, beta - h)) / (2 * h)
    assert gb == pytest.approx(fd, rel=1e-6)


def test_adjoint_config_512_matches_finite_differences():
    """The adjoint configuration's own grid: 512^2 periodic, seeded random
    velocity (E(k) ~ k^4 exp(-2 (k/8)^2), u_rms = 0.03, Re = 5000 on N), KBC B
    in FP64, 100 steps with checkpoints every 50; dJ/du0 of the final kinetic
    energy at three nodes and dJ/dbeta against central differences of the GPU
    forward map, h = 1e-6, agreement 1e-6 relative.  The difference of the
    two perturbed objectives is summed node by node (the nodes outside the
    perturbation's reach give identical bits), so the difference quotient
    carries no cancellation against the total energy."""
    n, steps, K = 512, 100, 50
    rho, ux, uy = flows.turbulence(n, k0=8, urms=0.03, seed=2024)
    beta = 1.0 / (6 * (n * 0.03 / 5000.0) + 1)
    J, g, gb = _gpu_adjoint("B", "f64", beta, rho, ux, uy, steps, K, 0)

    def ke_of(ux_, uy_, b):
        lat = Lattice(n, n, variant="B", beta=b, dtype="f64")
        lat.init(rho, ux_, uy_).step(steps)
        r, vx, vy = (t.cpu().numpy() for t in lat.moments())
        lat.close()
        return 0.5 * r * (vx * vx + vy * vy)

    assert J == pytest.approx(np.sum(ke_of(ux, uy, beta)), rel=1e-12)
    h = 1e-6
    for (yy, xx) in ((7, 400), (256, 256), (511, 0)):
        for comp in (0, 1):
            up, um = (ux.copy(), uy.copy()), (ux.copy(), uy.copy())
            up[comp][yy, xx] += h
            um[comp][yy, xx] -= h
            fd = np.sum(ke_of(*up, beta) - ke_of(*um, beta)) / (2 * h)
            assert g[comp, yy, xx] == pytest.approx(fd, rel=1e-6), (yy, xx, comp)
    fd = np.sum(ke_of(ux, uy, beta + h) - ke_of(ux, uy, beta - h)) / (2 * h)
    assert gb == pytest.approx(fd, rel=1e-6)


@pytest.mark.parametrize("dtype,guard", [("f64", None), ("f32", None), ("f32", 1e-10), ("f16", None)])
def test_checkpoint_interval_does_not_change_gradients(dtype, guard):
    """Recomputed segments are bit-identical to the forward sweep, so the
    gradients do not depend on the checkpoint interval.  Even intervals that
    fit the run (6, 10, 30) replay captured graphs of whole segments, several
    of them for 6 and 10, whose recompute changes the FP32 guard's counter
    parity from one segment to the next; odd ones (1, 7) and 100 launch step
    by step.  The guard at 1e-10 sends many nodes through the FP64
    re-evaluation every step, so that its counters carry real counts."""
    n, steps = 128, 30
    rho, ux, uy, tx, ty = _case(n, 3, k0=4.0)
    out = [_gpu_adjoint("B", dtype, 0.98, rho, ux, uy, steps, K, 0, guard=guard)
           for K in (1, 6, 7, 10, 30, 100)]
    for J, g, gb in out[1:]:
        assert J == out[0][0] and gb == out[0][2]
        assert np.array_equal(g, out[0][1])


def test_autograd_function_returns_adjoint_gradients():
    n, steps = 64, 20
    rho, ux, uy, tx, ty = _case(n, 4, k0=3.0)
    u0 = torch.tensor(np.stack((ux, uy)), device="cuda", requires_grad=True)
    beta = torch.tensor(0.96, dtype=torch.float64, requires_grad=True)
    tgt = torch.tensor(np.stack((tx, ty)), device="cuda")
    J = kbc_objective(u0, beta, rho0=torch.tensor(rho, device="cuda"), variant="B",
                      dtype="f64", steps=steps, ckpt_every=8, objective="misfit", u_target=tgt)
    (3.0 * J).backward()
    Jd, g, gb = _gpu_adjoint("B", "f64", 0.96, rho, ux, uy, steps, 8, 1, tx, ty)
    assert float(J.detach()) == Jd
    assert np.array_equal(u0.grad.cpu().numpy(), 3.0 * g)
    assert float(beta.grad) == pytest.approx(3.0 * gb, rel=1e-15)


@pytest.mark.parametrize("seed", [11, 13, 17])
def test_fp32_adjoint_tracks_fp64_on_512(seed):
    """Adjoint configuration: 512^2 periodic, seeded random velocity (k0 = 8),
    KBC B, 100 steps, checkpoints every 20; gradient of the final kinetic
    energy, FP32 storage/arithmetic against the FP64 adjoint.  Over seeds
    11-20 the FP32 error stays at the rounding level up to 100 steps (max
    norm <= 9.6e-4, L2 <= 2.6e-5, J <= 3.7e-9, dJ/dbeta <= 4.2e-7); beyond
    that the exact linearisation amplifies rounding where gamma* is poorly
    determined and the error becomes seed-dependent (seeds 13 and 17, taken
    here, are the first to leave: 0.08 and 0.13 at 200 steps)."""
    n, steps, K = 512, 100, 20
    rho, ux, uy = flows.turbulence(n, k0=8, urms=0.03, seed=seed)
    nu = n * 0.03 / 5000.0
    beta = 1.0 / (6 * nu + 1)
    J64, g64, gb64 = _gpu_adjoint("B", "f64", beta, rho, ux, uy, steps, K, 0)
    J32, g32, gb32 = _gpu_adjoint("B", "f32", beta, rho, ux, uy, steps, K, 0)
    rel_g = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    l2_g = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    print(f"512^2 {steps} steps, seed {seed}: J rel {abs(J32 - J64) / J64:.2e}, grad_u0 rel "
          f"{rel_g:.2e} (L2 {l2_g:.2e}), grad_beta rel {abs(gb32 - gb64) / abs(gb64):.2e}")
    assert abs(J32 - J64) <= 1e-7 * J64
    assert rel_g < 3e-3 and l2_g < 1e-4
    assert abs(gb32 - gb64) <= 1e-5 * abs(gb64)


def test_fp16_storage_adjoint_tracks_fp64():
    """FP16 storage (scaled half deviations, float arithmetic; the reverse
    step that loads node by node): J and the gradients of 20 steps on a
    128^2 field follow the FP64 adjoint to the storage's rounding level
    (measured: J 1.2e-5, dJ/du0 2.8e-4 in the max norm, dJ/dbeta 1.2e-5)."""
    n, steps, K = 128, 20, 10
    rho, ux, uy, _, _ = _case(n, 6, k0=4.0, urms=0.04)
    J64, g64, gb64 = _gpu_adjoint("B", "f64", 0.97, rho, ux, uy, steps, K, 0)
    J16, g16, gb16 = _gpu_adjoint("B", "f16", 0.97, rho, ux, uy, steps, K, 0)
    rel_g = np.max(np.abs(g16 - g64)) / np.max(np.abs(g64))
    print(f"f16 adjoint: J rel {abs(J16 - J64) / J64:.2e}, grad_u0 rel {rel_g:.2e}, "
          f"grad_beta rel {abs(gb16 - gb64) / abs(gb64):.2e}")
    assert abs(J16 - J64) <= 1e-4 * J64
    assert rel_g < 3e-3
    assert abs(gb16 - gb64) <= 1e-4 * abs(gb64)


def test_fp32_adjoint_overflow_is_reported():
    """Smooth 512^2 field (k0 = 1), KBC B, 300 steps: where <dh|dh> is tiny
    gamma* (Eq. result21) leaves [0, 2/beta], the linearised step amplifies
    by |1 - beta gamma| > 1 and the single-precision reverse sweep
    overflows.  The call reports KBC_ERR_NONFINITE instead of returning
    non-finite gradients as a success; the handle stays usable and the FP64
    adjoint of the same problem is finite."""
    n, steps, K = 512, 300, 30
    rho, ux, uy = flows.turbulence(n, k0=1, urms=0.03, seed=11)
    beta = 1.0 / (6 * (n * 0.03 / 5000.0) + 1)
    with pytest.raises(capi.KBCError) as ei:
        _gpu_adjoint("B", "f32", beta, rho, ux, uy, steps, K, 0)
    assert ei.value.status == capi.KBC_ERR_NONFINITE
    assert "adjoint" in str(ei.value)
    J, g, gb = _gpu_adjoint("B", "f64", beta, rho, ux, uy, steps, K, 0)
    assert np.isfinite(J) and np.isfinite(gb) and np.all(np.isfinite(g))


@pytest.mark.parametrize("variant", ["lbgk", "A", "B", "C", "D"])
@pytest.mark.parametrize("objective,fixed", [(0, False), (1, False), (0, True)])
def test_fp32_adjoint_tracks_fp64_all_models(variant, objective, fixed):
    """The single-precision reverse collision (opposite population pairs in
    packed FP32x2 lanes) against the double one on a 64^2 turbulent field,
    16 steps, every model, both objectives and the fixed-gamma mode.  The
    measured FP32 errors (J <= 2e-8, dJ/du0 <= 1.4e-3 in the max norm for A
    with the misfit objective and <= 1.4e-4 elsewhere, dJ/dbeta <= 8.1e-6)
    are those of the earlier one-population-at-a-time arithmetic; the bounds
    leave a factor of about 3."""
    n, steps, beta = 64, 16, 0.95
    rho, ux, uy = flows.turbulence(n, k0=4, urms=0.05, seed=3, kcut=16)
    rng = np.random.default_rng(4)
    tx = ux + 0.01 * rng.standard_normal(ux.shape)
    ty = uy + 0.01 * rng.standard_normal(uy.shape)
    gam = 1.0 / beta if fixed else None
    J64, g64, gb64 = _gpu_adjoint(variant, "f64", beta, rho, ux, uy, steps, 4, objective, tx, ty,
                                  gamma=gam)
    J32, g32, gb32 = _gpu_adjoint(variant, "f32", beta, rho, ux, uy, steps, 4, objective, tx, ty,
                                  gamma=gam)
    rel_g = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    assert abs(J32 - J64) <= 1e-7 * abs(J64)
    assert rel_g < 5e-3, rel_g
    assert abs(gb32 - gb64) <= 3e-5 * abs(gb64)
