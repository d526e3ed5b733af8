"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
the oracle on the same seeded inputs, and compare."""
import numpy as np

from paper_2305_05025_gb300 import lbmd, synth


def rel_linf(a, b):
    """max |a - b| / max |b| (0 when both are zero)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.abs(b).max() if b.size else 0.0
    num = np.abs(a - b).max() if b.size else 0.0
    return 0.0 if den == 0.0 and num == 0.0 else num / max(den, 1e-300)


def make(cfg, inp):
    h = lbmd.lbmd_create(cfg, inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    lbmd.lbmd_set_state(h, rho=inp["rho"].astype(np.float32), u=inp["u"].astype(np.float32),
                        x=inp["x"], v=inp["v"].astype(np.float32))
    return h


def oracle_start(orc, cfg, inp):
    """Oracle initial populations from the same (rho, u) the GPU got, rounded
    to FP32 first so both start from identical inputs."""
    rho = inp["rho"].astype(np.float32).astype(np.float64)
    u = inp["u"].astype(np.float32).astype(np.float64)
    f = orc.equilibrium(rho, u)
    topo = orc.Topology(inp["mass"], inp["bonds"], inp["bond_k"], inp["bond_r0"])
    return f, inp["x"].copy(), inp["v"].astype(np.float32).astype(np.float64), topo


def gpu_state(h):
    s = lbmd.lbmd_get_fields(h, f=True, rho=True, u=True, x=True, v=True)
    return s


def velocity(orc, cfg, f):
    """u = (sum f c + g/2)/rho of oracle populations."""
    rho, j = orc.moments(f)
    g = orc.body_force(cfg)
    return (j + 0.5 * g) / rho


def lattice_inputs(shape, sigma, seed, rho0=1.0):
    rho, u = synth.velocity_field(shape, sigma, seed, rho0)
    return dict(rho=rho, u=u, x=np.zeros((3, 0)), v=np.zeros((3, 0)), mass=np.zeros(0),
                bonds=np.zeros((0, 2), np.int32), bond_k=np.zeros(0), bond_r0=np.zeros(0))


HALF_ULP = 2.0 ** -24


def fp32_floor(orc, cfg, topo, f, x, v, steps, seed=0):
    """Relative L-infinity response of the FP64 oracle, after `steps` steps, to
    perturbing its inputs at the resolution the CUDA path stores them with:
    delta f and v by one FP32 half-ulp (relative), positions by one half-ulp of
    a unit cell offset (absolute). A CUDA result within this bound is as
    accurate as an exact computation from FP32-rounded inputs."""
    rng = np.random.default_rng(seed)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)[:, None] * cfg.get("rho0", 1.0)
    fp = w + (f - w) * (1 + rng.uniform(-HALF_ULP, HALF_ULP, f.shape))
    xp = x + rng.uniform(-HALF_ULP, HALF_ULP, x.shape)
    vp = v * (1 + rng.uniform(-HALF_ULP, HALF_ULP, v.shape))
    fa, xa, va, _ = orc.run(cfg, topo, f, x, v, steps)
    fb, xb, vb, _ = orc.run(cfg, topo, fp, xp, vp, steps)
    return dict(f=rel_linf(fb, fa), u=rel_linf(velocity(orc, cfg, fb), velocity(orc, cfg, fa)),
                x=rel_linf(xb, xa), v=rel_linf(vb, va)), (fa, xa, va)


def assert_within(errs, floors, tol=1e-5):
    """Each field within max(tol, its FP32 floor)."""
    for k, e in errs.items():
        bound = max(tol, floors.get(k, 0.0))
        assert e <= bound, f"{k}: error {e:.3e} > bound {bound:.3e} (floor {floors.get(k, 0.0):.3e})"
