"""Training checkpoint and resume (gmc_train_save_state / gmc_train_load_state):
a run stopped after k steps, saved, restored into a fresh training state and
continued ends where the uninterrupted run ends (bit for bit when two
uninterrupted runs agree bit for bit, else within their spread); malformed
checkpoints, a mismatched batch and a checkpoint saved on other data are
refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_resume_continues_the_run(gpu_ctx, kaiming_file, precision):
    import torch
    import paper_2512_13965_gb300 as g
    ctx = g.Context(0)
    try:
        g.gmc_load_weights(ctx, kaiming_file)
        n = 1 << 16
        cond = torch.empty(5, n, device="cuda")
        y = torch.empty(4, n, device="cuda")
        g.gmc_train_data(ctx, n, 3, 0.1, 1000.0, 0.5, 0.999, cond, y)
        torch.cuda.synchronize()
        cfg = g.gmc_train_config(batch=1024, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                                 weight_decay=0.01, seed=5,
                                 precision=g.GMC_BF16 if precision == "bf16" else g.GMC_FP32)
        P = g.gmc_train_param_count()

        def run(k1, k2, resume):
            g.gmc_train_begin(ctx, n, cond, y, cfg)
            g.gmc_train_steps(ctx, k1)
            g.gmc_train_set_lr(ctx, 5e-4)
            if resume:
                blob = g.gmc_train_save_state(ctx)
                assert len(blob) == g.gmc_train_state_size(ctx)
                g.gmc_train_begin(ctx, n, cond, y, cfg)  # step 0, initial weights, lr 1e-3
                g.gmc_train_load_state(ctx, blob)
            g.gmc_train_steps(ctx, k2)
            p = np.zeros(P, np.float32)
            g.gmc_train_params(ctx, p)
            return p

        a = run(4, 6, False)
        a2 = run(4, 6, False)
        b = run(4, 6, True)
        spread = float(np.abs(a - a2).max())
        if spread == 0.0:
            assert np.array_equal(a, b)
        else:
            assert np.abs(b - a).max() <= 10.0 * spread
        assert np.abs(a - run(0, 0, False)).max() > 1e-4  # the steps moved the weights

        blob = g.gmc_train_save_state(ctx)
        with pytest.raises(g.GMCError) as e:
            g.gmc_train_load_state(ctx, blob[:-4])
        assert e.value.status == g.GMC_EFORMAT
        bad = bytearray(blob)
        bad[0:4] = b"XXXX"
        with pytest.raises(g.GMCError) as e:
            g.gmc_train_load_state(ctx, bytes(bad))
        assert e.value.status == g.GMC_EFORMAT
        other = g.gmc_train_config(batch=512, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                                   weight_decay=0.01, seed=5)
        g.gmc_train_begin(ctx, n, cond, y, other)
        with pytest.raises(g.GMCError) as e:
            g.gmc_train_load_state(ctx, blob)
        assert e.value.status == g.GMC_EINVAL
        # the same batch and precision on other data: a smaller prefix of the
        # dataset (other n), then a dataset of the same size drawn with another seed
        half_c = cond[:, : n // 2].contiguous()
        half_y = y[:, : n // 2].contiguous()
        g.gmc_train_begin(ctx, n // 2, half_c, half_y, cfg)
        with pytest.raises(g.GMCError) as e:
            g.gmc_train_load_state(ctx, blob)
        assert e.value.status == g.GMC_EINVAL
        cond2 = torch.empty(5, n, device="cuda")
        y2 = torch.empty(4, n, device="cuda")
        g.gmc_train_data(ctx, n, 4, 0.1, 1000.0, 0.5, 0.999, cond2, y2)
        g.gmc_train_begin(ctx, n, cond2, y2, cfg)
        with pytest.raises(g.GMCError) as e:
            g.gmc_train_load_state(ctx, blob)
        assert e.value.status == g.GMC_EINVAL
        g.gmc_train_begin(ctx, n, cond, y, cfg)
        g.gmc_train_load_state(ctx, blob)  # the original data is accepted again
    finally:
        ctx.close()
