"""GPU analog random-walk transmission (analog_transmit) against the FP64
oracle walk and the walk's closed forms.

Both sides consume the same Philox counters, so most particles follow the
same path; the float position arithmetic of thin cells can still flip a
boundary decision, so tallies are compared within 4 standard errors and the
per-particle agreement only has to be high, not total.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(ctx, e, tau, c, mode, seed=0, id0=0, event0=0):
    import paper_2512_13965_gb300 as g
    n = e["xi"].shape[0]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    g.analog_transmit(ctx, n, d(e["xi"]), d(e["cos"]), d(e["sin"]), d(np.full(n, tau)),
                      d(np.full(n, c)), mode, seed, id0, event0, st, ex, nc)
    torch.cuda.synchronize()
    ex = ex.cpu().numpy().astype(np.float64)
    return {"status": st.cpu().numpy(), "p": ex[0], "ux": ex[1], "uy": ex[2], "s": ex[3],
            "ncoll": nc.cpu().numpy().view(np.uint32).astype(np.int64)}


def _orc(e, tau, c, mode, seed=0):
    n = e["xi"].shape[0]
    f64 = lambda a: np.asarray(a, dtype=np.float64)
    r = oracle.transport.transmit(f64(e["xi"]), f64(e["cos"]), f64(e["sin"]), np.full(n, tau),
                                  np.full(n, c), mode, seed)
    r["p"] = np.where(r["status"] == 0, r["face"] + r["q"], -1.0)
    return r


def _tallies(r):
    n = r["status"].shape[0]
    ex = r["status"] == 0
    face = np.where(ex, np.floor(r["p"]).clip(0, 3), -1)
    out = {"absorbed": (r["status"] == 1).astype(float)}
    for f, name in enumerate(("bottom", "right", "top", "reflected")):
        out[name] = (ex & (face == f)).astype(float)
    out["s"] = r["s"]
    return out


def _compare(a, b, names):
    n1, n2 = len(a[names[0]]), len(b[names[0]])
    for k in names:
        se = math.sqrt(a[k].var() / n1 + b[k].var() / n2)
        assert abs(a[k].mean() - b[k].mean()) <= 4 * se + 1e-12, (k, a[k].mean(), b[k].mean(), se)


def test_cell_config_analog(gpu_ctx):
    # tau = 1, c = 0.9, 1e5 particles entering the left face (uniform xi,
    # cosine-weighted direction), Philox seed 0.
    n = 100000
    e = synth.cell_entries(n, 0)
    import paper_2512_13965_gb300 as g
    rg = _gpu(gpu_ctx, e, 1.0, 0.9, g.GMC_ABSORB_ANALOG)
    ro = _orc(e, 1.0, 0.9, 0)
    ta, tb = _tallies(rg), _tallies(ro)
    _compare(ta, tb, ["absorbed", "bottom", "right", "top", "reflected", "s"])
    # transmitted + reflected + absorbed = 1 exactly
    assert sum(ta[k].sum() for k in ("absorbed", "bottom", "right", "top", "reflected")) == n
    # per-particle agreement
    same = (rg["status"] == ro["status"]) & (np.floor(rg["p"]) == np.floor(ro["p"]))
    assert same.mean() > 0.99
    close = same & (np.abs(rg["s"] - ro["s"]) < 1e-4 * (1 + ro["s"]))
    assert close.mean() > 0.99
    # 32-bin exit-position and exit-angle histograms
    exg, exo = rg["status"] == 0, ro["status"] == 0
    hg, _ = np.histogram(rg["p"][exg], bins=32, range=(0, 4))
    ho, _ = np.histogram(ro["p"][exo], bins=32, range=(0, 4))
    z = (hg - ho) / np.sqrt(np.maximum(hg + ho, 1))
    assert np.all(np.abs(z) < 4)

    def angle(r, ex):
        f = np.floor(r["p"][ex]).astype(int)
        nx = np.select([f == 1, f == 3], [1.0, -1.0], 0.0)
        ny = np.select([f == 2, f == 0], [1.0, -1.0], 0.0)
        cosn = r["ux"][ex] * nx + r["uy"][ex] * ny
        sinn = r["ux"][ex] * ny - r["uy"][ex] * nx
        return np.arctan2(sinn, cosn)
    ag, _ = np.histogram(angle(rg, exg), bins=32, range=(-np.pi / 2, np.pi / 2))
    ao, _ = np.histogram(angle(ro, exo), bins=32, range=(-np.pi / 2, np.pi / 2))
    assert np.all(np.abs((ag - ao) / np.sqrt(np.maximum(ag + ao, 1))) < 4)


@pytest.mark.parametrize("tau,c", [(0.1, 0.9), (10.0, 0.999), (100.0, 0.999)])
def test_implicit_mode_mean_path(gpu_ctx, tau, c):
    # GPU walk against the closed form E[s] = pi tau / 4 (also exercises the
    # FP64 position path for tau > 64) and against the oracle's tallies.
    import paper_2512_13965_gb300 as g
    n = 100000 if tau < 50 else 20000
    e = synth.cell_entries(n, 7)
    rg = _gpu(gpu_ctx, e, tau, c, g.GMC_ABSORB_IMPLICIT, seed=3)
    assert np.all(rg["status"] == 0)
    se = rg["s"].std() / math.sqrt(n)
    assert abs(rg["s"].mean() - math.pi * tau / 4) < 4 * se
    k = rg["ncoll"].astype(float)
    assert abs(k.mean() - c * math.pi * tau / 4) < 4 * k.std() / math.sqrt(n) + 1e-9
    if tau < 50:
        ro = _orc(e, tau, c, 1, seed=3)
        _compare(_tallies(rg), _tallies(ro), ["bottom", "right", "top", "reflected", "s"])


def test_pure_absorber_closed_form(gpu_ctx):
    import paper_2512_13965_gb300 as g
    from tests.test_oracle_walk import uncollided_by_face
    n, tau = 200000, 1.0
    e = synth.cell_entries(n, 11)
    rg = _gpu(gpu_ctx, e, tau, 0.0, g.GMC_ABSORB_ANALOG, seed=5)
    expect = uncollided_by_face(tau)
    face = np.floor(rg["p"])
    for f in range(3):
        p = np.mean((rg["status"] == 0) & (face == f))
        assert abs(p - expect[f]) < 4 * math.sqrt(expect[f] * (1 - expect[f]) / n)


def test_edge_sizes_and_errors(gpu_ctx):
    import paper_2512_13965_gb300 as g
    e = synth.cell_entries(1, 1)
    r = _gpu(gpu_ctx, e, 2.0, 0.5, g.GMC_ABSORB_ANALOG)
    assert r["status"][0] in (0, 1)
    z = torch.zeros(1, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    ex = torch.zeros(4, 1, device="cuda")
    g.analog_transmit(gpu_ctx, 0, z, z, z, z, z, 0, 0, 0, 0, st, ex)
    with pytest.raises(g.GMCError):
        g.analog_transmit(gpu_ctx, 1, z, z, z, z, z, 7, 0, 0, 0, st, ex)


def test_pinned_host_buffers_in_place(gpu_ctx):
    """Page-locked host arrays are read and written in place by the walk
    kernel: outputs equal those from device arrays bit for bit."""
    import paper_2512_13965_gb300 as g
    n = 20000 + 3
    e = synth.cell_entries(n, 77)
    ref = _gpu(gpu_ctx, e, 2.0, 0.9, g.GMC_ABSORB_IMPLICIT, seed=5)
    p = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).pin_memory()
    st = torch.full((n,), -7, dtype=torch.int32).pin_memory()
    ex = torch.full((4, n), float("nan")).pin_memory()
    nc = torch.zeros(n, dtype=torch.int32).pin_memory()
    g.analog_transmit(gpu_ctx, n, p(e["xi"]), p(e["cos"]), p(e["sin"]), p(np.full(n, 2.0)),
                      p(np.full(n, 0.9)), g.GMC_ABSORB_IMPLICIT, 5, 0, 0, st, ex, nc)
    exn = ex.numpy().astype(np.float64)
    assert np.array_equal(st.numpy(), ref["status"])
    assert np.array_equal(exn[0], ref["p"]) and np.array_equal(exn[3], ref["s"])
    assert np.array_equal(exn[1], ref["ux"]) and np.array_equal(exn[2], ref["uy"])
    assert np.array_equal(nc.numpy().view(np.uint32).astype(np.int64), ref["ncoll"])
