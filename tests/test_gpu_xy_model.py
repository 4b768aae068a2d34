"""The boundary model of x-y geometry on the GPU (3-D directions encoded by
their projection on the unit disk): its training data (gmc_train_data_xy)
against the oracle's 3-D walk on the same Philox counters, the sampler with
the unit-disk decode (gmc_transmit_xy) against the FP64 network and
oracle.mlp.decode_disk, and the gain of training over the untrained network
at held-out conditions, measured against the oracle's walk."""
import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import transport as T

pytestmark = pytest.mark.gpu


def _u01_f32(x):
    # the device's float uniform: fma((float)x, 2^-32, 2^-32)
    return (x.astype(np.float32) * np.float32(2.0 ** -32) + np.float32(2.0 ** -32)).astype(np.float32)


def _data(ctx, n, seed, tau=(0.1, 1000.0), c=(0.5, 0.999)):
    import paper_2512_13965_gb300 as g
    cond = torch.empty(5, n, device="cuda")
    y = torch.empty(4, n, device="cuda")
    g.gmc_train_data_xy(ctx, n, seed, tau[0], tau[1], c[0], c[1], cond, y)
    torch.cuda.synchronize()
    return cond, y


@pytest.fixture(scope="module")
def xctx(kaiming_file):
    import paper_2512_13965_gb300 as g
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, kaiming_file)
    g.gmc_load_xy_weights(ctx, kaiming_file)
    yield ctx
    ctx.close()


def test_xy_training_data_inputs_follow_philox(xctx):
    n, seed = 4096, 19
    cond, _ = _data(xctx, n, seed)
    c = cond.cpu().numpy().astype(np.float64)
    r0 = oracle.rng.philox_batch(seed, n, id0=0, event=0, tag=8)
    r1 = oracle.rng.philox_batch(seed, n, id0=0, event=1, tag=8)
    lo, hi = np.log(np.float32(0.1)), np.log(np.float32(1000.0))
    np.testing.assert_allclose(c[3], lo + (hi - lo) * _u01_f32(r0[:, 0]), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(c[4], 0.5 + (0.999 - 0.5) * _u01_f32(r0[:, 1]), rtol=1e-6)
    np.testing.assert_allclose(c[0], _u01_f32(r0[:, 2]), rtol=1e-7)
    mu = np.sqrt(_u01_f32(r0[:, 3]).astype(np.float64))
    np.testing.assert_allclose(c[1], mu, atol=1e-6)
    phi = 2.0 * np.pi * _u01_f32(r1[:, 0]).astype(np.float64)
    np.testing.assert_allclose(c[2], np.sqrt(1.0 - mu * mu) * np.cos(phi), atol=2e-6)
    assert np.all(c[1] ** 2 + c[2] ** 2 <= 1.0 + 1e-6) and np.all(c[1] > 0)


def test_xy_training_targets_match_oracle_walk(xctx):
    # the entries the kernel drew, the same counters (id i, flights from
    # event 2): the oracle's 3-D walk gives the same exits history by history
    n, seed = 20000, 23
    cond, y = _data(xctx, n, seed, tau=(0.3, 100.0))
    c = cond.cpu().numpy().astype(np.float64)
    yg = y.cpu().numpy().astype(np.float64)
    tau = np.exp(c[3])
    uz = np.sqrt(np.maximum(1.0 - c[1] ** 2 - c[2] ** 2, 0.0))
    r = T.transmit_xy(c[0], c[1], c[2], uz, tau, tau, c[4], T.MODE_IMPLICIT, seed,
                      ids=np.arange(n, dtype=np.uint64), events=np.full(n, 2, np.uint32))
    same = (np.floor(yg[0]) == r["face"]) & (np.abs(yg[3] - np.log(r["s"])) < 1e-3)
    assert same.mean() > 0.99
    assert np.abs(yg[0] - (r["face"] + r["q"]))[same].max() < 1e-3
    assert np.abs(yg[1] - r["ux"])[same].max() < 1e-4
    assert np.abs(yg[2] - r["uy"])[same].max() < 1e-4
    assert np.all(yg[1] ** 2 + yg[2] ** 2 <= 1.0 + 1e-5)


def test_xy_sampler_fp32_and_disk_decode(xctx, kaiming_file):
    import paper_2512_13965_gb300 as g
    net = oracle.mlp.read_weights(kaiming_file)
    n = 3000
    e = synth.cell_entries_xy(n, 81)
    tau, c = synth.materials(n, 82)
    cond = np.stack([e["xi"], e["ux"], e["uy"], np.log(tau), c]).astype(np.float32)
    z = synth.gaussian_noise(n, 83)
    y = torch.empty(4, n, device="cuda")
    ex = torch.empty(4, n, device="cuda")
    g.gmc_transmit_xy(xctx, n, torch.from_numpy(cond).cuda(), torch.from_numpy(z).cuda(), 0, 0, 8,
                      g.GMC_MIDPOINT, g.GMC_FP32, y, ex)
    torch.cuda.synchronize()
    yg = y.cpu().numpy().astype(np.float64)
    eg = ex.cpu().numpy().astype(np.float64)
    assert np.abs(yg - oracle.mlp.sample(net, cond, z, 8, "midpoint")).max() < 1e-4
    d = oracle.mlp.decode_disk(net, yg)
    dp = np.abs(eg[0] - (d["face"] + d["q"]))
    assert np.minimum(dp, 4.0 - dp).max() < 1e-4
    assert np.abs(eg[1] - d["ux"]).max() < 1e-4 and np.abs(eg[2] - d["uy"]).max() < 1e-4
    assert np.all(np.abs(eg[3] / d["s"] - 1.0) < 1e-4)
    # inside the disk, outward through the exit face
    assert np.all(eg[1] ** 2 + eg[2] ** 2 <= 1.0 + 1e-6)
    normal = np.array([[0, -1], [1, 0], [0, 1], [-1, 0]], np.float64)[d["face"]]
    assert np.all(eg[1] * normal[:, 0] + eg[2] * normal[:, 1] >= 0.0)
    # the same network through the square-cell slot decodes onto the circle
    ex2 = torch.empty(4, n, device="cuda")
    g.gmc_transmit(xctx, n, torch.from_numpy(cond).cuda(), torch.from_numpy(z).cuda(), 0, 0, 8,
                   g.GMC_MIDPOINT, g.GMC_FP32, None, ex2)
    torch.cuda.synchronize()
    e2 = ex2.cpu().numpy()
    np.testing.assert_allclose(e2[1] ** 2 + e2[2] ** 2, 1.0, atol=1e-5)


def test_xy_training_gain(xctx, tmp_path):
    # train on x-y walk data; the trained network's exits are closer (1-D
    # Wasserstein distance per output) to the oracle's 3-D walk at held-out
    # conditions than the untrained network's
    import paper_2512_13965_gb300 as g
    n = 1 << 20
    cond, y = _data(xctx, n, 5)
    cfg = g.gmc_train_config(batch=8192, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                             weight_decay=0.01, seed=11)
    g.gmc_train_begin(xctx, n, cond, y, cfg)
    steps = 600
    losses = np.zeros(steps, np.float32)
    g.gmc_train_steps(xctx, steps, losses)
    assert np.all(np.isfinite(losses)) and losses[-50:].mean() < 0.8 * losses[:20].mean()

    def exits(tau, cc, m=20000):
        e = synth.cell_entries_xy(m, 77)
        cnd = np.stack([e["xi"], e["ux"], e["uy"], np.full(m, np.log(tau)), np.full(m, cc)])
        ex = torch.empty(4, m, device="cuda")
        g.gmc_transmit_xy(xctx, m, torch.from_numpy(cnd.astype(np.float32)).cuda(), None, 5, 0, 16,
                          g.GMC_EULER, g.GMC_BF16, None, ex)
        torch.cuda.synchronize()
        return ex.cpu().numpy().astype(np.float64), e

    pairs = [(0.5, 0.9), (3.0, 0.99), (30.0, 0.75)]
    before = {p: exits(*p)[0] for p in pairs}
    path = str(tmp_path / "trained_xy.bin")
    g.gmc_train_commit(xctx, path)
    g.gmc_load_xy_weights(xctx, path)
    for tau, cc in pairs:
        after, e = exits(tau, cc)
        m = after.shape[1]
        ux, uy = e["ux"].astype(np.float32).astype(np.float64), e["uy"].astype(np.float32).astype(np.float64)
        uz = np.sqrt(np.maximum(1.0 - ux * ux - uy * uy, 0.0))
        r = T.transmit_xy(e["xi"].astype(np.float32).astype(np.float64), ux, uy, uz,
                          np.full(m, tau), np.full(m, tau), np.full(m, cc), T.MODE_IMPLICIT, 99)
        ref = [r["face"] + r["q"], r["ux"], r["uy"], np.log(r["s"])]
        for k in range(4):
            b = before[(tau, cc)][k] if k != 3 else np.log(before[(tau, cc)][3])
            a = after[k] if k != 3 else np.log(after[3])
            assert oracle.stats.w1(a, ref[k]) < oracle.stats.w1(b, ref[k]), (tau, cc, k)
