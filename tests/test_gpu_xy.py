"""GPU random walk in x-y geometry (analog_transmit_xy: 3-D directions given
and returned by their projection on the unit disk) against the closed forms
and the FP64 oracle (oracle.transport.transmit_xy) on the same Philox
counters."""
import math

import numpy as np
import pytest
import torch
from scipy import special

import synth
from oracle import transport as T

pytestmark = pytest.mark.gpu


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _entries(n, seed):
    # the kernel reads float32: the oracle gets the same rounded entries and
    # the out-of-plane component they imply
    e = synth.cell_entries_xy(n, seed)
    xi, ux, uy = (e[k].astype(np.float32).astype(np.float64) for k in ("xi", "ux", "uy"))
    uz = np.sqrt(np.maximum(1.0 - ux * ux - uy * uy, 0.0))
    return xi, ux, uy, uz


def _xy(ctx, xi, ux, uy, tx, ty, c, mode, seed):
    import paper_2512_13965_gb300 as g
    n = xi.shape[0]
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    g.analog_transmit_xy(ctx, n, _d(xi), _d(ux), _d(uy), _d(np.full(n, tx)), _d(np.full(n, ty)),
                         _d(np.full(n, c)), mode, seed, 0, 0, st, ex, nc)
    torch.cuda.synchronize()
    x = ex.cpu().numpy().astype(np.float64)
    return {"status": st.cpu().numpy(), "p": x[0], "ux": x[1], "uy": x[2], "s": x[3],
            "ncoll": nc.cpu().numpy()}


@pytest.mark.parametrize("tx,ty,c", [(2.0, 0.5, 0.9), (100.0, 3.0, 0.95)])
def test_matches_oracle(gpu_ctx, tx, ty, c):
    # same entries and counters; float against double positions can flip a
    # decision now and then, so the laws are compared within 4 sigma and
    # nearly every history must agree
    n = 20000
    xi, ux, uy, uz = _entries(n, 501)
    r = _xy(gpu_ctx, xi, ux, uy, tx, ty, c, 1, 6)
    o = T.transmit_xy(xi, ux, uy, uz, np.full(n, tx), np.full(n, ty), np.full(n, c),
                      T.MODE_IMPLICIT, 6)
    face = np.floor(r["p"]).astype(int)
    for f in range(4):
        a, b = np.mean(face == f), np.mean(o["face"] == f)
        assert abs(a - b) < 4 * math.sqrt(max(b * (1 - b), 1.0 / n) / n) + 1e-9, (f, a, b)
    assert abs(r["s"].mean() - o["s"].mean()) < 4 * o["s"].std() / math.sqrt(n)
    same = np.abs(r["s"] - o["s"]) < 1e-3 * np.maximum(o["s"], 1.0)
    assert same.mean() > 0.99, same.mean()
    assert np.mean(r["ncoll"] == o["ncoll"]) > 0.99
    for k in ("ux", "uy"):
        assert np.abs(r[k] - o[k])[same].max() < 1e-3, k


def test_mean_track_square_prism(gpu_ctx):
    # Cauchy's 4 A / P at any scattering ratio: tau for the square
    n, tau = 1 << 20, 2.0
    xi, ux, uy, _ = _entries(n, 502)
    r = _xy(gpu_ctx, xi, ux, uy, tau, tau, 0.9, 1, 7)
    assert (r["status"] == 0).all()
    assert abs(r["s"].mean() - tau) < 4 * r["s"].std() / math.sqrt(n)
    k = r["ncoll"] - 0.9 * r["s"]
    assert abs(k.mean()) < 4 * k.std() / math.sqrt(n)


def test_slab_uncollided_transmission(gpu_ctx):
    # a cell far taller than wide (FP64 positions) with every collision
    # absorbing: the right-face fraction is 2 E3(tx)
    n, tx = 1 << 20, 0.3
    xi, ux, uy, _ = _entries(n, 503)
    r = _xy(gpu_ctx, xi, ux, uy, tx, 1e6 * tx, 0.0, 0, 8)
    face = np.floor(r["p"]).astype(int)
    p = np.mean((r["status"] == 0) & (face == 1))
    expect = 2.0 * special.expn(3, tx)
    assert abs(p - expect) < 4 * math.sqrt(expect * (1 - expect) / n), (p, expect)


def test_exit_projection_in_disk_and_outward(gpu_ctx):
    n = 1 << 16
    xi, ux, uy, _ = _entries(n, 504)
    r = _xy(gpu_ctx, xi, ux, uy, 1.7, 0.9, 0.8, 1, 9)
    ok = r["status"] == 0
    assert ok.all()
    assert (np.hypot(r["ux"], r["uy"]) <= 1.0 + 1e-6).all()
    face = np.floor(r["p"]).astype(int)
    outward = np.array([[0.0, -1.0], [1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]])[face]
    assert (r["ux"] * outward[:, 0] + r["uy"] * outward[:, 1] > 0.0).all()


def test_errors(gpu_ctx):
    import paper_2512_13965_gb300 as g
    x = _d(np.zeros(2))
    st = torch.empty(2, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, 2, device="cuda")
    with pytest.raises(g.GMCError) as err:
        g.analog_transmit_xy(gpu_ctx, 2, x, x, x, x, x, x, 7, 0, 0, 0, st, ex)
    assert err.value.status == g.GMC_EINVAL
    with pytest.raises(g.GMCError) as err:
        g.analog_transmit_xy(gpu_ctx, 2, x, None, x, x, x, x, 1, 0, 0, 0, st, ex)
    assert err.value.status == g.GMC_EINVAL
