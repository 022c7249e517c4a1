"""What the trained FNO gains over the method without it, on small cropped blocks (16^3 crops of the
128x128x256 dipping-TI model at 400 kHz; the full-size run is ``python -m
paper_2306_17537_gb300.fno_warmstart``).

The network is trained by the library's own kernels on blocks solved by the library, then every
held-out block is solved cold (E := b) and warm (E := b + FNO prediction) to the same FP64 residual.
Measured and asserted: the trained prediction is accepted by ie_solve's fallback rule on most blocks and
lowers the initial residual e (eq. 9) several-fold; the warm solves reach the same tolerance; an
untrained network (zero output, i.e. E := b) is rejected, so the gain comes from training. The GMRES
iteration counts of both modes are reported; on these high-contrast blocks they are set by the slow
part of the convergence and change little.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_fno_lowers_the_initial_residual_of_held_out_blocks(capsys):
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import fno_warmstart as fw
    from paper_2306_17537_gb300 import ie, inputs

    n, n_train, n_test = 16, 96, 12
    wl0 = inputs.config4_item(0, n)
    opts = fw.solve_opts(ie, 40, 4000, 4)
    with ie.Context(wl0.grid, wl0.grid.h, wl0.sigma0, wl0.freq) as ctx, \
            ie.FNO(n, modes=4, width=16, layers=4, hidden=32, batch_max=8, bf16=True) as net:
        # untrained: all-zero parameters predict E = b, which the fallback rule rejects
        net.set_params(np.zeros(net.param_count(), np.float32))
        test_models = list(fw.item_stream(range(n_train, n_train + n_test), n, 1))
        cold0 = fw.compare(torch, ie, net, ctx, wl0, test_models[:3], 1e-6, opts)
        assert cold0["warm"]["used"] == 0
        net.set_params(fw.init_flat(ie, n, 4, 16, 4, 32, 0))
        data = fw.Data(torch, n_train, n)
        fw.generate(torch, ie, net, ctx, wl0, fw.item_stream(range(n_train), n, 1), data, 1e-6, opts)
        train_idx = np.flatnonzero(data.ok)
        curve, _, _ = fw.train(torch, net, data, train_idx, 8, 25, 2e-3)
        assert curve[-1] < 0.7 * curve[0]
        cmp = fw.compare(torch, ie, net, ctx, wl0, test_models, 1e-6, opts)
    cold, warm = cmp["cold"], cmp["warm"]
    ratio = np.array(warm["initial_e_warm"]) / np.array(warm["initial_e_cold"])
    with capsys.disabled():
        print(f"\nFNO warm start on {n_test} held-out 16^3 blocks: train loss {curve[0]:.3f} -> {curve[-1]:.3f}, "
              f"median initial-residual ratio {np.median(ratio):.3f}, accepted {warm['used']}/{n_test}, "
              f"mean GMRES iterations cold {cold['mean_iters']:.1f} warm {warm['mean_iters']:.1f}")
    assert warm["used"] >= n_test * 3 // 4
    assert np.median(ratio) < 0.5
    assert warm["solved"] == cold["solved"] >= n_test - 2
    assert warm["max_e_solved"] <= 1e-6 and cold["max_e_solved"] <= 1e-6
