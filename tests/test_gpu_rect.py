"""GPU random walk in rectangular cells (analog_transmit_rect, the geometry
variant with unequal sides) against the square walk, the closed forms and
the FP64 oracle (oracle.transport.transmit_rect)."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import transport as T
from test_oracle_rect import uncollided_rect

pytestmark = pytest.mark.gpu


def _d(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rect(ctx, e, tx, ty, c, mode, seed=0):
    import paper_2512_13965_gb300 as g
    n = e["xi"].shape[0]
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    g.analog_transmit_rect(ctx, n, _d(e["xi"]), _d(e["cos"]), _d(e["sin"]), _d(np.full(n, tx)),
                           _d(np.full(n, ty)), _d(np.full(n, c)), mode, seed, 0, 0, st, ex, nc)
    torch.cuda.synchronize()
    x = ex.cpu().numpy().astype(np.float64)
    return {"status": st.cpu().numpy(), "p": x[0], "ux": x[1], "uy": x[2], "s": x[3],
            "ncoll": nc.cpu().numpy()}


@pytest.mark.parametrize("tau,c,mode", [(0.7, 0.9, 1), (3.0, 0.6, 0), (80.0, 0.95, 1)])
def test_equal_sides_is_the_square_walk(gpu_ctx, tau, c, mode):
    import paper_2512_13965_gb300 as g
    n = 20000
    e = synth.cell_entries(n, 401)
    r = _rect(gpu_ctx, e, tau, tau, c, mode, seed=3)
    st = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    nc = torch.empty(n, dtype=torch.int32, device="cuda")
    g.analog_transmit(gpu_ctx, n, _d(e["xi"]), _d(e["cos"]), _d(e["sin"]), _d(np.full(n, tau)),
                      _d(np.full(n, c)), mode, 3, 0, 0, st, ex, nc)
    torch.cuda.synchronize()
    x = ex.cpu().numpy().astype(np.float64)
    assert np.array_equal(r["status"], st.cpu().numpy())
    assert np.array_equal(r["ncoll"], nc.cpu().numpy())
    for k, row in (("p", 0), ("ux", 1), ("uy", 2), ("s", 3)):
        assert np.array_equal(r[k], x[row]), k


@pytest.mark.parametrize("tx,ty", [(2.0, 0.5), (0.5, 3.0)])
def test_uncollided_closed_form(gpu_ctx, tx, ty):
    n = 1 << 20
    e = synth.cell_entries(n, 402)
    r = _rect(gpu_ctx, e, tx, ty, 0.0, 0)
    expect = uncollided_rect(tx, ty)
    face = np.floor(r["p"]).astype(int)
    for f in range(3):
        p = np.mean((r["status"] == 0) & (face == f))
        se = math.sqrt(max(expect[f] * (1 - expect[f]), 1e-12) / n)
        assert abs(p - expect[f]) < 4 * se + 1e-9, (f, p, expect[f])


@pytest.mark.parametrize("tx,ty,c", [(2.0, 0.5, 0.9), (100.0, 3.0, 0.95)])
def test_matches_oracle(gpu_ctx, tx, ty, c):
    # same entries and Philox counters; float against double positions can
    # flip a decision now and then, so the laws are compared within 4 sigma
    n = 20000
    e = synth.cell_entries(n, 403)
    r = _rect(gpu_ctx, e, tx, ty, c, 1, seed=6)
    o = T.transmit_rect(e["xi"], e["cos"], e["sin"], np.full(n, tx), np.full(n, ty),
                        np.full(n, c), T.MODE_IMPLICIT, 6)
    face = np.floor(r["p"]).astype(int)
    for f in range(4):
        a, b = np.mean(face == f), np.mean(o["face"] == f)
        assert abs(a - b) < 4 * math.sqrt(max(b * (1 - b), 1.0 / n) / n) + 1e-9, (f, a, b)
    assert abs(r["s"].mean() - o["s"].mean()) < 4 * o["s"].std() / math.sqrt(n)
    same = np.mean(np.abs(r["s"] - o["s"]) < 1e-3 * np.maximum(o["s"], 1.0))
    assert same > 0.99, same


def test_errors(gpu_ctx):
    import paper_2512_13965_gb300 as g
    x = _d(np.zeros(2))
    st = torch.empty(2, dtype=torch.int32, device="cuda")
    ex = torch.empty(4, 2, device="cuda")
    with pytest.raises(g.GMCError) as err:
        g.analog_transmit_rect(gpu_ctx, 2, x, x, x, x, x, x, 7, 0, 0, 0, st, ex)
    assert err.value.status == g.GMC_EINVAL
