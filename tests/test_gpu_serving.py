"""Serving: continuous batching of transport solves (gmc_serve_start /
gmc_submit / gmc_poll / gmc_wait). A request's flux is the same alone, in a
mix with other requests, and from transport_solve; admission respects the
memory budget."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _grid(n, seed, tau_hi=20.0):
    tau, c, src = synth.grid_problem(n=n, seed=seed, tau_range=(0.1, tau_hi), block=max(n // 4, 1),
                                     source=max(n // 8, 1))
    return (np.ascontiguousarray(tau.ravel()), np.ascontiguousarray(c.ravel()),
            np.ascontiguousarray(src.ravel()))


@pytest.fixture
def server_ctx(kaiming_file):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    g.gmc_load_weights(ctx, kaiming_file)
    cfg = g.gmc_get_config(ctx)
    cfg.bank_capacity = 1 << 16
    cfg.steps = 8
    g.gmc_set_config(ctx, cfg)
    yield ctx
    g.gmc_serve_stop(ctx)
    ctx.close()


@pytest.mark.parametrize("method", [0, 1])
def test_alone_equals_mix_equals_transport_solve(server_ctx, method):
    import paper_2512_13965_gb300 as g
    ctx = server_ctx
    A = _grid(16, 3)
    n_a = 30000
    # transport_solve reference
    ref = np.zeros(256)
    g.transport_solve(ctx, 16, 16, *A, n_a, method, 77, ref)
    g.gmc_serve_start(ctx, method, 64 << 20)
    # alone
    fa = np.zeros(256)
    t = g.gmc_submit(ctx, 16, 16, *A, n_a, 77)
    st_alone = g.gmc_wait(ctx, t, 120.0, fa)
    # in a mix of requests of other sizes submitted around it
    others = []
    for k, n in enumerate((8, 32, 24, 16)):
        G = _grid(n, 10 + k)
        others.append((n, g.gmc_submit(ctx, n, n, *G, 20000 + 5000 * k, 500 + k)))
    fm = np.zeros(256)
    t2 = g.gmc_submit(ctx, 16, 16, *A, n_a, 77)
    for n, tk in others[:2]:
        g.gmc_wait(ctx, tk, 120.0, np.zeros(n * n))
    st_mix = g.gmc_wait(ctx, t2, 120.0, fm)
    for n, tk in others[2:]:
        g.gmc_wait(ctx, tk, 120.0, np.zeros(n * n))
    np.testing.assert_allclose(fa, ref, rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(fm, ref, rtol=1e-9, atol=1e-15)
    assert st_alone.transmissions == st_mix.transmissions
    assert st_mix.latency > 0 and st_alone.latency > 0


def test_admission_by_memory(server_ctx):
    import paper_2512_13965_gb300 as g
    ctx = server_ctx
    # 64x64 grids need ~98 KiB each; a 1 MiB budget holds ~10 at a time
    g.gmc_serve_start(ctx, 0, 1 << 20)
    big = _grid(256, 5)
    with pytest.raises(g.GMCError) as e:
        g.gmc_submit(ctx, 256, 256, *big, 1000, 1)
    assert e.value.status == g.GMC_ENOMEM
    tickets = []
    for k in range(24):
        G = _grid(64, 100 + k, tau_hi=5.0)
        tickets.append(g.gmc_submit(ctx, 64, 64, *G, 3000, 900 + k))
    seen_busy = False
    results = {}
    deadline = time.time() + 180
    while len(results) < len(tickets) and time.time() < deadline:
        for tk in tickets:
            if tk in results:
                continue
            f = np.zeros(64 * 64)
            st = g.gmc_poll(ctx, tk, f)
            if st is None:
                seen_busy = True
            else:
                results[tk] = (f, st)
        time.sleep(0.001)
    assert len(results) == len(tickets)
    assert seen_busy
    for f, st in results.values():
        assert np.all(np.isfinite(f)) and f.sum() > 0
        assert abs(st.absorbed + st.leaked - st.roulette_net - 3000) < 1e-3 * 3000
    with pytest.raises(g.GMCError):
        g.gmc_poll(ctx, tickets[0], np.zeros(64 * 64))  # retired ticket
