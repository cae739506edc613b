"""Shared helpers of the GPU parity tests (input preparation only)."""
import numpy as np

import oracle as O

W = None


def weights():
    global W
    if W is None:
        W = O.weights()
    return W


def representable(f, dtype: str, f16_scale: float = 1.0):
    """Round populations f[9][ny][nx] to what the given storage holds exactly.

    Storage keeps d = f - W_i (f64, f32) or (f - W_i)/W_i * S (f16); the
    rounding is applied on the host so that the oracle starts from the very
    values the GPU field holds.
    """
    Wb = weights().reshape(9, *([1] * (f.ndim - 1)))
    d = f - Wb
    if dtype == "f64":
        return f.copy()
    if dtype == "f32":
        return d.astype(np.float32).astype(np.float64) + Wb
    if dtype == "f16":
        h = (d * ((1.0 / Wb) * f16_scale)).astype(np.float16).astype(np.float64)
        return h * (Wb * (1.0 / f16_scale)) + Wb
    raise ValueError(dtype)


def random_field(nx, ny, seed, amp=0.02, umax=0.08):
    """Near-equilibrium populations with random rho, u and non-equilibrium part."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.02 * rng.standard_normal((ny, nx))
    ux = umax * (2 * rng.random((ny, nx)) - 1)
    uy = umax * (2 * rng.random((ny, nx)) - 1)
    g = O.init_feq(rho, ux, uy)
    g = g * (1.0 + amp * rng.standard_normal(g.shape))
    return g


def max_rel_velocity_error(u_gpu, u_ref):
    """max |u_gpu - u_ref| / max |u_ref| over both components."""
    (ax, ay), (bx, by) = u_gpu, u_ref
    num = max(np.max(np.abs(ax - bx)), np.max(np.abs(ay - by)))
    den = max(np.max(np.abs(bx)), np.max(np.abs(by)))
    return num / den


def windows(g0_fn, nx, ny, nodes_xy, steps, variant, beta, half=None, **kw):
    """Oracle populations at selected nodes after `steps` steps, each computed
    on its own periodic window of width 2*steps+1 (+2) around the node: the
    node's state after n steps depends only on the (2n+1)^2 box around it.

    g0_fn(xs, ys) returns the initial populations [9][len(ys)][len(xs)] on the
    index grid (xs, ys) of the full field.
    """
    half = steps + 1 if half is None else half
    out = []
    for (x, y) in nodes_xy:
        xs = (np.arange(x - half, x + half + 1)) % nx
        ys = (np.arange(y - half, y + half + 1)) % ny
        g = g0_fn(xs, ys)
        g = O.step(g, variant, beta, steps, **kw)
        out.append(g[:, half, half])
    return np.array(out)


def oracle_sensitivity(g0, variant, beta, steps, nthreads=16, seed=0, ref_uv=None, **kw):
    """Relative velocity gap between the oracle run from g0 and from g0 with
    every population perturbed by at most one ulp (seeded).  No FP64
    implementation of the same method can be expected to agree with the
    oracle more closely than this rounding-sensitivity floor.  kw: gamma
    mode arguments of O.step."""
    rng = np.random.default_rng(seed)
    gp = g0 * (1.0 + np.finfo(np.float64).eps * rng.choice([-1.0, 0.0, 1.0], size=g0.shape))
    b = O.step(gp, variant, beta, steps, nthreads=nthreads, **kw)
    _, bx, by = O.macro(b)
    if ref_uv is None:
        a = O.step(g0, variant, beta, steps, nthreads=nthreads, **kw)
        _, ax, ay = O.macro(a)
    else:
        ax, ay = ref_uv
    return max_rel_velocity_error((bx, by), (ax, ay))
