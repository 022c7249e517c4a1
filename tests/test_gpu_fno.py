"""FNO warm-start kernels (include/ie_fno.h) against the FP64 reference oracle/fno.py.

Forward output and every parameter gradient are compared per tensor in relative L2: 1e-4 with FP32
activation storage (FP32 accumulation of sums over up to n^3 terms), 2e-2 with BF16 storage (8-bit
mantissa of the stored activations and spectral weights). One Adam step is checked against its closed
form for the first step (update = lr g / (|g| + eps)). The warm-start encoding is checked against its
definition, and ie_solve's initial-guess hook against the cold start.
"""
import numpy as np
import pytest

from oracle import fno as ofno

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available()
    from paper_2306_17537_gb300 import ie

    return torch, ie


CASES = {
    # n, modes, width, layers, cin, cout, hidden, batch
    "tiny": (8, 3, 4, 2, 3, 2, 5, 2),
    "warmstart-shape": (16, 4, 8, 3, 12, 6, 16, 2),
    "ragged": (12, 5, 6, 2, 12, 6, 7, 3),
    # widths where the BF16 pointwise maps run on the tensor cores (the layers' 32 -> 32, the head's
    # 32 -> 128 and 128 -> 6 maps; the lift, 12 -> 32, stays on the CUDA cores)
    "tensor-core": (16, 4, 32, 2, 12, 6, 128, 3),
}


def _setup(case, seed):
    n, m, width, layers, cin, cout, hidden, B = CASES[case]
    rng = np.random.default_rng(seed)
    prm = ofno.init_params(seed, cin=cin, width=width, cout=cout, hidden=hidden, layers=layers, n=n, modes=m)
    prm.p = rng.normal(size=prm.p.shape) * 0.1
    prm.w = [rng.normal(size=w.shape) * 0.1 for w in prm.w]
    prm.q1 = rng.normal(size=prm.q1.shape) * 0.1
    prm.q2 = rng.normal(size=prm.q2.shape) * 0.1
    # spectral weights large enough that K_l matters against W_l
    prm.R = [r * width for r in prm.R]
    a = rng.normal(size=(B, n, n, n, cin))
    t = rng.normal(size=(B, n, n, n, cout))
    return prm, a, t


def _rel(x, y):
    x, y = np.asarray(x).ravel(), np.asarray(y).ravel()
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


def _net(ie, case, bf16):
    n, m, width, layers, cin, cout, hidden, B = CASES[case]
    return ie.FNO(n, modes=m, width=width, layers=layers, cin=cin, cout=cout, hidden=hidden, batch_max=B, bf16=bf16)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("bf16", [False, True])
def test_forward_and_gradients_match_oracle(env, case, bf16):
    torch, ie = env
    prm, a, t = _setup(case, 3)
    B = a.shape[0]
    u_ref, cache = ofno.forward(prm, a, keep=True)
    _, du = ofno.rel_l2_loss(u_ref, t)
    g_ref = ofno.backward(prm, cache, du)
    tol = 2e-2 if bf16 else 1e-4
    with _net(ie, case, bf16) as net:
        flat = ie.fno_flat(prm.flat())
        assert flat.size == net.param_count()
        net.set_params(flat)
        assert np.array_equal(net.get_params(), flat)
        dev = torch.device("cuda", 0)
        a_d = torch.from_numpy(a.astype(np.float32)).to(dev)
        u_d = torch.empty(u_ref.shape, dtype=torch.float32, device=dev)
        net.forward(B, a_d, u_d)
        torch.cuda.synchronize()
        assert _rel(u_d.cpu().numpy(), u_ref) <= tol
        du_d = torch.from_numpy(du.astype(np.float32)).to(dev)
        g = net.backward(B, a_d, du_d)
    off = 0
    for name, ref in zip(["P", "p"] + [f"W{l}" for l in range(len(prm.W))] + [f"w{l}" for l in range(len(prm.w))]
                         + [f"R{l}" for l in range(len(prm.R))] + ["Q1", "q1", "Q2", "q2"], ie_flat_parts(g_ref)):
        got = g[off: off + ref.size]
        off += ref.size
        assert _rel(got, ref) <= tol, (name, _rel(got, ref))
    assert off == g.size


def test_tensor_core_maps_match_cuda_core_maps(env):
    # the same BF16 network forward with the pointwise maps on the tcgen05 tensor cores and on the CUDA
    # cores: they differ only by the BF16 rounding of the weights the tensor cores read (and the order
    # of the FP32 sums), so the outputs agree to BF16 precision; both agree with the FP64 oracle
    torch, ie = env
    prm, a, _ = _setup("tensor-core", 5)
    B = a.shape[0]
    u_ref = ofno.forward(prm, a)
    dev = torch.device("cuda", 0)
    a_d = torch.from_numpy(a.astype(np.float32)).to(dev)
    outs = {}
    with _net(ie, "tensor-core", True) as net:
        net.set_params(ie.fno_flat(prm.flat()))
        for on in (False, True, True):  # the tensor-core path twice: it is deterministic
            net.set_tensor_cores(on)
            u_d = torch.full(u_ref.shape, float("nan"), dtype=torch.float32, device=dev)
            net.forward(B, a_d, u_d)
            torch.cuda.synchronize()
            outs.setdefault(on, []).append(u_d.cpu().numpy())
    cuda_core, tc = outs[False][0], outs[True][0]
    assert np.all(np.isfinite(tc))
    assert np.array_equal(outs[True][0], outs[True][1])
    assert _rel(tc, cuda_core) <= 1e-2
    assert _rel(tc, u_ref) <= 2e-2 and _rel(cuda_core, u_ref) <= 2e-2


def ie_flat_parts(prm):
    out = []
    for arr in prm.flat():
        a = np.asarray(arr)
        if np.iscomplexobj(a):
            a = np.stack([a.real, a.imag], axis=-1)
        out.append(a.ravel())
    return out


def test_train_step_is_one_adam_step_on_the_relative_l2_loss(env):
    torch, ie = env
    prm, a, t = _setup("warmstart-shape", 5)
    B = a.shape[0]
    u_ref, cache = ofno.forward(prm, a, keep=True)
    loss_ref, du = ofno.rel_l2_loss(u_ref, t)
    g_ref = np.concatenate(ie_flat_parts(ofno.backward(prm, cache, du)))
    lr = 1e-3
    with _net(ie, "warmstart-shape", False) as net:
        flat = ie.fno_flat(prm.flat())
        net.set_params(flat)
        dev = torch.device("cuda", 0)
        a_d = torch.from_numpy(a.astype(np.float32)).to(dev)
        t_d = torch.from_numpy(t.astype(np.float32)).to(dev)
        loss = net.train_step(B, a_d, t_d, lr)
        new = net.get_params()
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    # first Adam step: m/(1-b1) = g, v/(1-b2) = g^2  ->  step = lr g / (|g| + eps)
    big = np.abs(g_ref) > 1e-3 * np.max(np.abs(g_ref))
    expect = flat - lr * g_ref / (np.abs(g_ref) + 1e-8)
    assert np.max(np.abs(new[big] - expect[big])) <= 1e-3 * lr + 1e-6


def test_warm_start_encoding_matches_its_definition(env):
    torch, ie = env
    from paper_2306_17537_gb300 import inputs

    n = 16
    g = inputs.centred_grid(n, n, n, 0.25)
    s6 = inputs.random_contrast_sigma6((n, n, n), 2, 0.1)
    rng = np.random.default_rng(4)
    b = rng.normal(size=(3, n, n, n)) + 1j * rng.normal(size=(3, n, n, n))
    E = b + 0.3 * (rng.normal(size=b.shape) + 1j * rng.normal(size=b.shape))
    dev = torch.device("cuda", 0)
    with _net(ie, "warmstart-shape", True) as net:
        s6_d = torch.from_numpy(np.ascontiguousarray(s6)).to(dev)
        b_d = torch.from_numpy(b).to(dev)
        E_d = torch.from_numpy(E).to(dev)
        a_d = torch.empty((n ** 3, 12), dtype=torch.float32, device=dev)
        t_d = torch.empty((n ** 3, 6), dtype=torch.float32, device=dev)
        bn_d = torch.empty(1, dtype=torch.float64, device=dev)
        x0_d = torch.empty_like(b_d)
        net.encode(s6_d, 0.1, b_d, a_d, bn_d)
        net.encode_target(E_d, b_d, bn_d, t_d)
        net.decode(t_d, b_d, bn_d, x0_d)
        torch.cuda.synchronize()
        a_h, t_h, bn, x0 = a_d.cpu().numpy(), t_d.cpu().numpy(), float(bn_d.item()), x0_d.cpu().numpy()
    bnorm = np.linalg.norm(b)
    assert abs(bn - bnorm) <= 1e-12 * bnorm
    sc = np.sqrt(n ** 3) / bnorm
    ds = s6.reshape(-1, 6) - np.array([0.1, 0.1, 0.1, 0, 0, 0])
    bb = np.stack([b.reshape(3, -1).real, b.reshape(3, -1).imag], axis=-1).transpose(1, 0, 2).reshape(-1, 6) * sc
    assert np.allclose(a_h[:, :6], ds, rtol=1e-6, atol=1e-7)
    assert np.allclose(a_h[:, 6:], bb, rtol=1e-6, atol=1e-6)
    d = E - b
    tt = np.stack([d.reshape(3, -1).real, d.reshape(3, -1).imag], axis=-1).transpose(1, 0, 2).reshape(-1, 6) * sc
    assert np.allclose(t_h, tt, rtol=1e-6, atol=1e-6)
    # decode(encode_target(E)) = E up to the FP32 rounding of the target
    assert _rel(x0, E) <= 1e-6


def test_initial_guess_hook_uses_a_good_guess_and_rejects_a_bad_one(env):
    torch, ie = env
    from paper_2306_17537_gb300 import inputs

    wl = inputs.config2(0, scale=8)  # 16x16x32, 2 blocks
    dev = torch.device("cuda", 0)
    opts = ie.make_opts(restart=40, max_inner=4000, max_outer=60)
    with ie.Context(wl.grid, wl.grid.h, wl.sigma0, wl.freq) as ctx:
        ctx.set_contrast(wl.sigma6)
        H0, info0, _ = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-6, opts)
        E = torch.empty((3, wl.grid.nz, wl.grid.ny, wl.grid.nx), dtype=torch.complex128, device=dev)
        ctx.get_field_dev(E)
        # the converged field as the guess: accepted, and far fewer iterations than the cold start
        ctx.set_initial_field_dev(E)
        H1, info1, _ = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-6, opts)
        assert info1.warm_start_used == 1 and info1.warm_rel_residual < 1e-5 < info1.cold_rel_residual
        assert info1.gmres_iters_total < info0.gmres_iters_total // 4
        assert np.max(np.abs(H1 - H0)) <= 1e-5 * np.max(np.abs(H0))
        # a guess worse than E0 is rejected: the solve repeats the cold start exactly
        ctx.set_initial_field_dev(E * 50.0)
        H2, info2, _ = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-6, opts)
        assert info2.warm_start_used == 0 and info2.warm_rel_residual > info2.cold_rel_residual
        assert info2.gmres_iters_total == info0.gmres_iters_total
        assert np.array_equal(H2, H0)
        # the guess is consumed: the next solve is a plain cold start
        H3, info3, _ = ctx.solve(wl.sources, wl.receivers, ie.IE_DD_NONE, 1e-6, opts)
        assert info3.cold_rel_residual == 0.0 and info3.gmres_iters_total == info0.gmres_iters_total
