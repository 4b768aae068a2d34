"""Seeded synthetic inputs for the tests and the benchmark.

This module only draws inputs (cell entries, materials, noise, random network
weights) and writes them in the agreed formats. It holds none of the method's
arithmetic, and both the CUDA path's callers and the oracle's callers consume
what it returns. Random numbers come from numpy's Philox bit generator keyed
by the seed.

Workload recipes (the paper's geometries and data are not available, so each
input is drawn from the distributions the workload names):
  * cell entries: xi ~ U[0,1), sin(theta) ~ U(-1,1) (an inward direction with
    cosine-weighted density on the entry face), cos(theta) = sqrt(1 - sin^2);
  * x-y geometry entries: xi ~ U[0,1), the cosine to the face normal is
    sqrt(U[0,1)) and the azimuth about it U[0, 2 pi) (3-D cosine law);
  * sampler conditions: tau log-uniform in [0.1, 1000], c uniform in
    [0.5, 0.999], entries as above; condition vector
    (xi, cos theta, sin theta, ln tau, c);
  * network: 25 -> 256 -> 256 -> 256 -> 256 -> 4, weights Kaiming-normal
    N(0, 2 / fan_in), zero biases, identity standardization;
  * grid: n x n cells, tau log-uniform in [0.1, 500], c drawn from
    {0.5, 0.999} per 16 x 16 block, unit source spread over the central 8 x 8
    cells;
  * the paper's two benchmarks with their printed cross sections (lattice
    and linearized hohlraum, 112 x 112 meshes); their layouts are only in
    figures that are not available, so the arrangements are stand-ins.
"""
import struct

import numpy as np

DIMS = (25, 256, 256, 256, 256, 4)


def generator(seed):
    return np.random.Generator(np.random.Philox(key=int(seed)))


def cell_entries(n, seed):
    """Entry states on the left face: dict of float32 arrays xi, cos, sin."""
    g = generator(seed)
    xi = g.random(n)
    sn = g.uniform(-1.0, 1.0, n)
    cs = np.sqrt(np.maximum(1.0 - sn * sn, 0.0))
    return {"xi": xi.astype(np.float32), "cos": cs.astype(np.float32),
            "sin": sn.astype(np.float32)}


def cell_entries_xy(n, seed):
    """Entry states on the left face with 3-D directions (x-y geometry):
    xi ~ U[0,1), cosine to the face normal ux = sqrt(U[0,1)) (the cosine-law
    inflow of an isotropic flux), azimuth about the normal U[0, 2 pi):
    dict of float64 arrays xi, ux, uy, uz."""
    g = generator(seed)
    xi = g.random(n)
    mu = np.sqrt(g.random(n))
    phi = g.uniform(0.0, 2.0 * np.pi, n)
    r = np.sqrt(np.maximum(1.0 - mu * mu, 0.0))
    return {"xi": xi, "ux": mu, "uy": r * np.cos(phi), "uz": r * np.sin(phi)}


def materials(n, seed, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """tau log-uniform and c uniform, float32."""
    g = generator(seed)
    lo, hi = np.log(tau_range[0]), np.log(tau_range[1])
    tau = np.exp(g.uniform(lo, hi, n))
    c = g.uniform(c_range[0], c_range[1], n)
    return tau.astype(np.float32), c.astype(np.float32)


def sampler_conditions(n, seed, tau_range=(0.1, 1000.0), c_range=(0.5, 0.999)):
    """Condition vectors [5, n] float32: (xi, cos, sin, ln tau, c); plus tau and c."""
    e = cell_entries(n, seed)
    tau, c = materials(n, seed + 7919, tau_range, c_range)
    cond = np.stack([e["xi"], e["cos"], e["sin"], np.log(tau).astype(np.float32), c])
    return np.ascontiguousarray(cond, dtype=np.float32), tau, c


def gaussian_noise(n, seed):
    """Standard normal draws [4, n] float32."""
    return np.ascontiguousarray(generator(seed).standard_normal((4, n)), dtype=np.float32)


def kaiming_weights(seed=1):
    """Kaiming-normal weights (fan-in), zero biases, identity standardization."""
    g = generator(seed)
    W, b = [], []
    for l in range(5):
        fan_in, fan_out = DIMS[l], DIMS[l + 1]
        W.append((g.standard_normal((fan_out, fan_in)) * np.sqrt(2.0 / fan_in)).astype(np.float32))
        b.append(np.zeros(fan_out, dtype=np.float32))
    return {"W": W, "b": b, "cond_mean": np.zeros(5, np.float32), "cond_std": np.ones(5, np.float32),
            "y_mean": np.zeros(4, np.float32), "y_std": np.ones(4, np.float32)}


def kaiming_weights_rect(seed=1):
    """Kaiming-normal weights of the network for rectangular cells: 26
    inputs (the aspect component ln(tau_y / tau_x) as input column 25), zero
    biases, identity standardization of the 6 condition components."""
    net = kaiming_weights(seed)
    g = generator(seed + 3000)
    net["W"][0] = (g.standard_normal((256, 26)) * np.sqrt(2.0 / 26)).astype(np.float32)
    net["cond_mean"] = np.zeros(6, np.float32)
    net["cond_std"] = np.ones(6, np.float32)
    return net


def rect_conditions(n, seed, tau_range=(0.1, 1000.0), aspect_range=(0.25, 4.0),
                    c_range=(0.5, 0.999)):
    """Conditions of rectangular cells [6, n] float32: (xi, cos, sin,
    ln tau_x, c, ln(tau_y / tau_x)), tau_x log-uniform, the aspect
    tau_y / tau_x log-uniform in aspect_range, entries as cell_entries."""
    e = cell_entries(n, seed)
    tau, c = materials(n, seed + 7919, tau_range, c_range)
    g = generator(seed + 104729)
    la = g.uniform(np.log(aspect_range[0]), np.log(aspect_range[1]), n)
    cond = np.stack([e["xi"], e["cos"], e["sin"], np.log(tau).astype(np.float32), c,
                     la.astype(np.float32)])
    return np.ascontiguousarray(cond, dtype=np.float32)


def rm_weights(seed=1, m_std=0.0, g_std=0.0, base=None):
    """Weights of the residual-modulated network: the layers of `base` (default
    `kaiming_weights(seed)`), condition shifts M[3][256][5] ~ N(0, m_std^2)
    and channel scales G[3][2][256] ~ N(0, g_std^2) (zero by default: a
    training start whose blocks are unmodulated)."""
    net = dict(base if base is not None else kaiming_weights(seed))
    g = generator(seed + 2000)
    net["M"] = [(g.standard_normal((256, 5)) * m_std).astype(np.float32) for _ in range(3)]
    net["G"] = [(g.standard_normal((2, 256)) * g_std).astype(np.float32) for _ in range(3)]
    return net


def biased_weights(seed=7, bias_std=0.3):
    """Kaiming-normal weights with N(0, bias_std^2) biases and a non-identity
    standardization (condition and output means and standard deviations of
    the size a trained network's data statistics have)."""
    net = kaiming_weights(seed)
    g = generator(seed + 1000)
    net["b"] = [(g.standard_normal(len(b)) * bias_std).astype(np.float32) for b in net["b"]]
    net["cond_mean"] = g.uniform(-1.0, 1.0, 5).astype(np.float32)
    net["cond_std"] = g.uniform(0.5, 2.0, 5).astype(np.float32)
    net["y_mean"] = g.uniform(-0.5, 0.5, 4).astype(np.float32)
    net["y_std"] = g.uniform(0.3, 1.5, 4).astype(np.float32)
    return net


def write_weights(path, net):
    """Write a dict like `kaiming_weights()` returns as a GMCW version-1 file;
    with keys "M" and "G" (`rm_weights()`) flag 1 and those arrays follow the
    layers: M[3][256][5], then G[3][2][256]."""
    rm = "M" in net
    n_cond = len(net["cond_mean"])  # 6: a network for rectangular cells
    with open(path, "wb") as f:
        f.write(b"GMCW")
        f.write(struct.pack("<2I", 1, 5))
        f.write(struct.pack("<6I", n_cond + 20, *DIMS[1:]))
        f.write(struct.pack("<4I", n_cond, 4, 16, 1 if rm else 0))
        for k in ("cond_mean", "cond_std", "y_mean", "y_std"):
            f.write(np.asarray(net[k], dtype="<f4").tobytes())
        for l in range(5):
            f.write(np.ascontiguousarray(net["W"][l], dtype="<f4").tobytes())
            f.write(np.ascontiguousarray(net["b"][l], dtype="<f4").tobytes())
        if rm:
            for m in net["M"]:
                f.write(np.ascontiguousarray(m, dtype="<f4").reshape(256, 5).tobytes())
            for q in net["G"]:
                f.write(np.ascontiguousarray(q, dtype="<f4").reshape(2, 256).tobytes())


def grid_problem(n=128, seed=2, tau_range=(0.1, 500.0), c_values=(0.5, 0.999), block=16,
                 source=8):
    """Heterogeneous n x n grid: tau [n,n], c [n,n], src [n,n] (float32, row = y index)."""
    g = generator(seed)
    lo, hi = np.log(tau_range[0]), np.log(tau_range[1])
    tau = np.exp(g.uniform(lo, hi, (n, n)))
    nb = (n + block - 1) // block
    pick = g.integers(0, len(c_values), (nb, nb))
    cb = np.asarray(c_values, dtype=np.float64)[pick]
    c = np.kron(cb, np.ones((block, block)))[:n, :n]
    src = np.zeros((n, n))
    a = max((n - source) // 2, 0)
    src[a:a + source, a:a + source] = 1.0
    src /= src.sum()
    return tau.astype(np.float32), c.astype(np.float32), src.astype(np.float32)


# Material classes of the hohlraum-like boundary-source problem: (tau, c).
HOHLRAUM_MATERIALS = {"gas": (0.2, 1.0), "wall": (200.0, 0.6), "window": (0.5, 1.0),
                      "ablator": (20.0, 0.9), "fuel": (2.0, 0.99)}


def hohlraum_problem(n=64):
    """Hohlraum-like boundary-source problem on n x n unit cells with five
    material classes (HOHLRAUM_MATERIALS): a wall frame n/16 cells thick, open
    on the left between rows n/4 and 3n/4 (the entrance hole, filled with the
    window material); a capsule of radius n/6 at the centre (an ablator shell
    two cells thick around the fuel); gas elsewhere. The source drives the
    entrance hole from the left boundary. Returns tau [n, n], c [n, n]
    (float32, row = y index) and the left-boundary strengths wall [n]."""
    t = max(1, n // 16)
    lo, hi = n // 4, (3 * n) // 4
    ii, jj = np.meshgrid(np.arange(n), np.arange(n))  # ii: x index, jj: y index
    mat = np.full((n, n), "gas", dtype=object)
    frame = (jj < t) | (jj >= n - t) | (ii >= n - t) | (ii < t)
    mat[frame] = "wall"
    mat[(ii < t) & (jj >= lo) & (jj < hi)] = "window"
    r = np.hypot(ii + 0.5 - n / 2.0, jj + 0.5 - n / 2.0)
    R = n / 6.0
    mat[r < R] = "ablator"
    mat[r < R - 2.0] = "fuel"
    tau = np.vectorize(lambda m: HOHLRAUM_MATERIALS[m][0])(mat).astype(np.float32)
    c = np.vectorize(lambda m: HOHLRAUM_MATERIALS[m][1])(mat).astype(np.float32)
    wall = np.zeros(n, dtype=np.float32)
    wall[lo:hi] = 1.0
    return tau, c, wall



# Cross sections (sigma_a, sigma_s) in cm^-1 of the paper's benchmarks
# (section "Benchmark Performance"). Each cell of side h gets tau = sigma_t h
# and c = sigma_s / sigma_t.
LATTICE_XS = {"background": (0.0, 1.0), "absorber": (9.5, 0.5)}
PAPER_HOHLRAUM_XS = {"wall": (50.0, 50.0), "stripe": (5.0, 95.0), "frame": (10.0, 90.0),
                     "absorber": (95.0, 5.0), "vacuum": (0.0, 5.0)}


def _optical(xs, mat, h):
    sa = np.vectorize(lambda m: xs[m][0])(mat)
    ss = np.vectorize(lambda m: xs[m][1])(mat)
    st = sa + ss
    return (st * h).astype(np.float32), (ss / st).astype(np.float32)


def paper_lattice_problem(n=112):
    """The lattice benchmark's materials on a 7 x 7 cm square, n x n cells
    (n a multiple of 7): scattering background, absorbers (LATTICE_XS) and an
    isotropic volumetric source in the central 1 x 1 cm square. The absorber
    arrangement (a periodic array in the paper, whose figure is not
    available) is a stand-in: the 1 x 1 cm squares (a, b) of the inner 5 x 5
    with a + b even, the source square (3, 3) excepted. Returns tau, c, src
    [n, n] (float32, row = y index; src sums to 1)."""
    if n % 7:
        raise ValueError("n must be a multiple of 7")
    u = n // 7
    a = np.arange(n) // u
    A, B = np.meshgrid(a, a)  # A: x square, B: y square
    mat = np.full((n, n), "background", dtype=object)
    inner = (A >= 1) & (A <= 5) & (B >= 1) & (B <= 5)
    mat[inner & ((A + B) % 2 == 0) & ~((A == 3) & (B == 3))] = "absorber"
    tau, c = _optical(LATTICE_XS, mat, 7.0 / n)
    src = ((A == 3) & (B == 3)).astype(np.float64)
    return tau, c, (src / src.sum()).astype(np.float32)


def paper_hohlraum_problem(n=112):
    """The linearized hohlraum's materials on a 1.3 x 1.3 cm square, n x n
    cells (PAPER_HOHLRAUM_XS), driven by an isotropic surface source over the
    whole left boundary. The arrangement (in a figure that is not available)
    is a stand-in, mirror-symmetric about y = 0.65 cm: absorbing walls along
    the top, bottom and right (0.1 cm thick); stripes covering the left
    boundary outside the entrance 0.4 < y < 0.9 cm (0.1 cm thick); a square
    absorber of half-width 0.2 cm at the centre inside a frame 0.1 cm wide;
    near-vacuum elsewhere. Returns tau, c [n, n] (float32, row = y index)
    and the left-boundary strengths wall [n]."""
    h = 1.3 / n
    x = (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(x, x)
    mat = np.full((n, n), "vacuum", dtype=object)
    d = np.maximum(np.abs(X - 0.65), np.abs(Y - 0.65))
    mat[d < 0.3] = "frame"
    mat[d < 0.2] = "absorber"
    mat[(X < 0.1) & ((Y < 0.4) | (Y > 0.9))] = "stripe"
    mat[(X > 1.2) | (Y < 0.1) | (Y > 1.2)] = "wall"
    tau, c = _optical(PAPER_HOHLRAUM_XS, mat, h)
    return tau, c, np.ones(n, dtype=np.float32)
