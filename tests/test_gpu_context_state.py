"""Context state across calls: a weight load that fails leaves the network
loaded before in place (sampling and the training start both see it), and
while the server runs, reconfiguring or loading weights is refused with
GMC_EBUSY and changes nothing."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_failed_reload_keeps_the_loaded_network(gpu_ctx, kaiming_file, tmp_path):
    import torch
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, kaiming_file)
        n = 1024
        cond, _, _ = synth.sampler_conditions(n, 5)
        z = synth.gaussian_noise(n, 6)

        def sample():
            y = np.zeros((4, n), np.float32)
            g.gmc_transmit(ctx, n, cond, z, 0, 0, 4, g.GMC_EULER, g.GMC_FP32, y, None)
            return y

        y_before = sample()
        other = tmp_path / "biased.bin"
        synth.write_weights(str(other), synth.biased_weights())
        blob = other.read_bytes()
        with pytest.raises(g.GMCError) as e:
            g.gmc_load_weights_buffer(ctx, blob[:-4])  # last bias cut short
        assert e.value.status == g.GMC_EFORMAT
        assert np.array_equal(sample(), y_before)
        # training starts from the loaded network, not from the parsed part
        # of the rejected file
        m = 4096
        cd = torch.rand(5, m, device="cuda")
        yd = torch.rand(4, m, device="cuda")
        cfg = g.gmc_train_config(batch=1024, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                                 weight_decay=0.01, seed=1)
        g.gmc_train_begin(ctx, m, cd, yd, cfg)
        p = np.zeros(g.gmc_train_param_count(), np.float32)
        g.gmc_train_params(ctx, p)
        net = synth.kaiming_weights(1)
        assert np.array_equal(p[:256 * 32].reshape(256, 32)[:, :25], net["W"][0])
        o = 256 * 32 + 256
        assert np.array_equal(p[o:o + 65536].reshape(256, 256), net["W"][1])
    finally:
        ctx.close()


def test_running_server_refuses_reconfiguration(gpu_ctx, kaiming_file):
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, kaiming_file)
        cfg = g.gmc_get_config(ctx)
        cfg.bank_capacity = 1 << 16
        g.gmc_set_config(ctx, cfg)
        steps0 = cfg.steps
        g.gmc_serve_start(ctx, g.GMC_METHOD_ANALOG, 1 << 20)
        cfg2 = g.gmc_get_config(ctx)
        cfg2.steps = steps0 + 1
        with pytest.raises(g.GMCError) as e:
            g.gmc_set_config(ctx, cfg2)
        assert e.value.status == g.GMC_EBUSY
        assert "server" in str(e.value)
        for load in (g.gmc_load_weights, g.gmc_load_internal_weights):
            with pytest.raises(g.GMCError) as e:
                load(ctx, kaiming_file)
            assert e.value.status == g.GMC_EBUSY
        assert g.gmc_get_config(ctx).steps == steps0
        g.gmc_serve_stop(ctx)
        g.gmc_set_config(ctx, cfg2)
        assert g.gmc_get_config(ctx).steps == steps0 + 1
        g.gmc_load_internal_weights(ctx, kaiming_file)
    finally:
        ctx.close()
