"""The surrogate's tensor-core kernels against the fp64 oracle (oracle/
mlp_oracle.py, which rounds weights and activations to BF16 as the network
stores them): forward outputs, parameter gradients, the MSE loss, AdamW; then
training convergence and a small end-to-end surrogate of the simulator.

Tolerances: the GPU accumulates in FP32 and rounds each activation to BF16; a
pre-activation that differs from the fp64 value by FP32 rounding can land in
the neighbouring BF16 step (2^-8 relative), so outputs and gradients are
compared by relative norm at 1e-2 and element-wise at a few BF16 steps."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sur():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_03235_b300 import surrogate
    return surrogate


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("B", [300, 64, 1])
def test_forward_and_gradients_match_oracle(sur, B):
    import torch
    net = sur.MLP(seed=5, max_batch=512)
    rng = np.random.default_rng(B)
    x = rng.normal(size=(B, 16)).astype(np.float32)
    xb = torch.as_tensor(x).cuda().to(torch.bfloat16)
    y = net.forward(xb).double().cpu().numpy()
    p = net.params.double().cpu().numpy()
    want, _ = M.forward(list(sur.DIMS), p, x)
    assert rel(y, want) < 1e-2
    assert np.allclose(y, want, rtol=3e-2, atol=3e-2 * np.abs(want).max())
    dy = rng.normal(size=(B, 16)).astype(np.float32)
    g = net.backward(xb, torch.as_tensor(dy).cuda()).double().cpu().numpy()
    gw = M.backward(list(sur.DIMS), p, x, dy.astype(np.float64))
    off = 0
    for l in range(len(sur.DIMS) - 1):
        n, k = sur.DIMS[l + 1], sur.DIMS[l]
        for size in (n * k, n):
            a, b = g[off:off + size], gw[off:off + size]
            assert rel(a, b) < 2e-2, (l, size)
            off += size


def test_mse_and_adamw_match_oracle(sur):
    import torch
    net = sur.MLP(seed=1, max_batch=128)
    rng = np.random.default_rng(7)
    y = rng.normal(size=(100, 16)).astype(np.float32)
    t = rng.normal(size=(100, 16)).astype(np.float32)
    loss, dy = net.mse(torch.as_tensor(y).cuda(), torch.as_tensor(t).cuda(), 3)
    wl, wdy = M.mse(y, t, 3)
    assert abs(loss.item() - wl) < 1e-5 * wl
    assert np.allclose(dy.cpu().numpy(), wdy, rtol=1e-5, atol=1e-9)
    p = net.params.double().cpu().numpy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in range(1, 4):
        g = rng.normal(size=p.size).astype(np.float32)
        net.grads.copy_(torch.as_tensor(g))
        net.adamw(1e-3, wd=0.01)
        p, m, v = M.adamw(p, g.astype(np.float64), m, v, 1e-3, 0.9, 0.999, 1e-8, 0.01, step)
    got = net.params.double().cpu().numpy()
    assert np.allclose(got, p, rtol=1e-5, atol=1e-6)
    assert np.array_equal(net.params_bf16.float().cpu().numpy(),
                          M.bf16_round(net.params.cpu().numpy()).astype(np.float32))


def test_training_fits_a_smooth_function(sur):
    import torch
    s = sur.Surrogate(seed=3, max_batch=1024)
    rng = np.random.default_rng(0)
    X = np.zeros((4096, 16), dtype=np.float32)
    X[:, :10] = rng.uniform(-1, 1, size=(4096, 10))
    Y = np.stack([np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2], X[:, 3] ** 2 - X[:, 4],
                  np.exp(0.5 * X[:, 5])], axis=1)
    first = s.fit(X, Y, epochs=1, batch=512, lr=2e-3)
    last = s.fit(X, Y, epochs=60, batch=512, lr=2e-3)
    assert last < 0.1 * first
    pred = s.predict(X[:512])
    assert np.abs(pred - Y[:512]).mean() < 0.1


def test_small_surrogate_of_the_simulator_and_screening(sur):
    """Train on simulated design points, score on fresh simulations, and show
    what screening with the network gains over random screening at the same
    simulation budget (the lowest mean L2 access latency found)."""
    kw = dict(sides=(8, 16, 24), period_lo=2, period_hi=40)
    X, Y, _ = sur.make_dataset(600, 3000, seed=1, **kw)
    s = sur.Surrogate(seed=0, max_batch=1024)
    s.fit(X, Y, epochs=150, batch=128, lr=2e-3)
    Xh, Yh, _ = sur.make_dataset(100, 3000, seed=2, **kw)
    err = sur.relative_errors(s.predict(Xh), Yh)
    assert err.mean(axis=0).max() < 0.35
    # screening: 400 candidates, simulate 10 chosen by the network vs 10 random
    Xc, _, pc = sur.make_dataset(400, 1, seed=3, **kw)
    pred = s.predict(Xc)
    top = np.argsort(pred[:, 0])[:10]
    rnd = np.random.default_rng(9).choice(400, size=10, replace=False)
    y_top = sur.simulate([pc[i] for i in top], 3000)
    y_rnd = sur.simulate([pc[i] for i in rnd], 3000)
    assert y_top[:, 0].min() < y_rnd[:, 0].min()


@pytest.mark.parametrize("B", [128, 1024])
def test_tcgen05_layer_exact_sum(sur, B):
    """One 256 -> 256 layer at a batch the tcgen05 path takes: the result is
    the fp64 sum of the BF16 products to FP32 accuracy, on both GEMM engines."""
    import torch
    net = sur.MLP(dims=(256, 256), seed=11, max_batch=B)
    rng = np.random.default_rng(B)
    x = rng.normal(size=(B, 256)).astype(np.float32)
    xb = torch.as_tensor(x).cuda().to(torch.bfloat16)
    p = M.bf16_round(net.params.double().cpu().numpy())
    W, b = p[:256 * 256].reshape(256, 256), p[256 * 256:]
    want = M.bf16_round(x) @ W.T + b
    out = {}
    for path in (0, 1):
        old = sur.set_gemm_path(path)
        out[path] = net.forward(xb).double().cpu().numpy()
        sur.set_gemm_path(old)
    assert sur.gemm_status() == 0
    scale = np.abs(want).max()
    for path in (0, 1):
        assert np.abs(out[path] - want).max() < 2e-5 * scale, path
    assert np.abs(out[0] - out[1]).max() < 2e-5 * scale


@pytest.mark.parametrize("B", [128, 4096])
def test_tcgen05_network_matches_mma_sync_and_oracle(sur, B):
    """The full network (three 256 x 256 hidden layers on tcgen05 at these
    batches) against the mma.sync engine and the fp64 oracle."""
    import torch
    net = sur.MLP(seed=7, max_batch=B)
    rng = np.random.default_rng(B + 1)
    x = rng.normal(size=(B, 16)).astype(np.float32)
    xb = torch.as_tensor(x).cuda().to(torch.bfloat16)
    old = sur.set_gemm_path(1)
    y1 = net.forward(xb).double().cpu().numpy()
    sur.set_gemm_path(0)
    y0 = net.forward(xb).double().cpu().numpy()
    sur.set_gemm_path(old)
    assert sur.gemm_status() == 0
    want, _ = M.forward(list(sur.DIMS), net.params.double().cpu().numpy(), x)
    assert rel(y0, want) < 1e-2
    assert np.allclose(y0, want, rtol=3e-2, atol=3e-2 * np.abs(want).max())
    assert rel(y0, y1) < 5e-3


def _grads_both_paths(sur, net, xb, dy):
    import torch
    out = {}
    for path in (0, 1):
        old = sur.set_gemm_path(path)
        net.forward(xb)
        out[path] = net.backward(xb, torch.as_tensor(dy).cuda()).double().cpu().numpy()
        sur.set_gemm_path(old)
    assert sur.gemm_status() == 0
    return out


@pytest.mark.parametrize("B", [1024, 256])
def test_tcgen05_backward_matches_mma_sync_and_oracle(sur, B):
    """At training batches the tcgen05 path takes the backward GEMMs too: the
    weight gradients (a contraction over the batch, in chunks of 256) on K-major
    transposes of dZ and the layer input, the input gradients on W^T.  Both
    engines accumulate in FP32, so they agree to FP32 rounding; both match the
    fp64 oracle to BF16 accuracy."""
    import torch
    net = sur.MLP(seed=13, max_batch=B)
    rng = np.random.default_rng(B + 5)
    x = rng.normal(size=(B, 16)).astype(np.float32)
    xb = torch.as_tensor(x).cuda().to(torch.bfloat16)
    dy = rng.normal(size=(B, 16)).astype(np.float32)
    g = _grads_both_paths(sur, net, xb, dy)
    p = net.params.double().cpu().numpy()
    gw = M.backward(list(sur.DIMS), p, x, dy.astype(np.float64))
    off = 0
    for l in range(len(sur.DIMS) - 1):
        n, k = sur.DIMS[l + 1], sur.DIMS[l]
        for size in (n * k, n):
            a0, a1, want = g[0][off:off + size], g[1][off:off + size], gw[off:off + size]
            assert rel(a0, a1) < 1e-4, (l, size)
            assert rel(a0, want) < 2e-2, (l, size)
            off += size


def test_tcgen05_long_contraction(sur):
    """A 512 -> 256 layer at batch 512: the forward GEMM (K = 512, two chunks
    of the tcgen05 kernel's K loop) against the mma.sync engine and the exact
    fp64 sum of the BF16 products; its weight gradient (512 columns, wider
    than the tcgen05 tile allows, so on mma.sync under either setting) against
    the same sum."""
    import torch
    B = 512
    net = sur.MLP(dims=(512, 256), seed=17, max_batch=B)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(B, 512)).astype(np.float32)
    xb = torch.as_tensor(x).cuda().to(torch.bfloat16)
    p = M.bf16_round(net.params.double().cpu().numpy())
    W, b = p[:512 * 256].reshape(256, 512), p[512 * 256:]
    want = M.bf16_round(x) @ W.T + b
    ys = {}
    for path in (0, 1):
        old = sur.set_gemm_path(path)
        ys[path] = net.forward(xb).double().cpu().numpy()
        sur.set_gemm_path(old)
    scale = np.abs(want).max()
    for path in (0, 1):
        assert np.abs(ys[path] - want).max() < 2e-5 * scale, path
    dy = rng.normal(size=(B, 256)).astype(np.float32)
    g = _grads_both_paths(sur, net, xb, dy)
    gW = M.bf16_round(dy.astype(np.float64)).T @ M.bf16_round(x)
    for path in (0, 1):
        got = g[path][:512 * 256].reshape(256, 512)
        assert np.abs(got - gW).max() < 2e-5 * np.abs(gW).max(), path


@pytest.mark.parametrize("dims,B", [(None, 4096), (None, 128), ((64, 128, 256, 32), 384),
                                    ((16, 192, 64), 256)])
def test_fused_inference_equals_layered_forward(sur, dims, B):
    """The one-kernel inference (weights packed into the operand layout and
    brought in by bulk copies, activations kept on chip, TMEM accumulators
    chained layer to layer) gives exactly the layered tensor-core forward's
    outputs, which the tests above tie to the fp64 oracle; the image is
    repacked after a parameter update."""
    import torch
    net = sur.MLP(dims=dims or sur.DIMS, seed=21, max_batch=B)
    rng = np.random.default_rng(B)
    x = rng.normal(size=(B, net.dims[0])).astype(np.float32)
    xb = torch.as_tensor(x).cuda().to(torch.bfloat16)
    old = sur.set_gemm_path(0)
    y_layered = net.forward(xb).cpu().numpy()
    y_fused = net.infer(xb).cpu().numpy()
    assert sur.gemm_status() == 0
    assert np.array_equal(y_fused, y_layered)
    want, _ = M.forward(list(net.dims), net.params.double().cpu().numpy(), x)
    assert rel(y_fused.astype(np.float64), want) < 1e-2
    net.grads.copy_(torch.as_tensor(rng.normal(size=net.n).astype(np.float32)))
    net.adamw(1e-2)
    assert np.array_equal(net.infer(xb).cpu().numpy(), net.forward(xb).cpu().numpy())
    sur.set_gemm_path(old)
    with pytest.raises(ValueError):
        net.infer(xb[:64])
    # the C ABI refuses a batch that is not a multiple of 128 (MLP_ERR_ARG)
    import ctypes as C
    y = torch.empty(64, net.dims[-1], device="cuda")
    L = sur._mlp_lib()
    assert L.mlp_infer(C.byref(net.shape), net._packed(), sur._p(xb), 64, sur._p(y), net._stream()) == 1


def test_fused_inference_replays_in_a_cuda_graph(sur):
    """mlp_infer launched on the caller's stream captures into a CUDA graph:
    a replay writes into the captured output buffer exactly what a direct
    call gives, and a replay after the input buffer changes follows it."""
    import torch
    net = sur.MLP(seed=5, max_batch=4096)
    xb = torch.rand(4096, sur.DIMS[0], device="cuda").to(torch.bfloat16)
    y = torch.empty(4096, sur.DIMS[-1], device="cuda")
    net.infer(xb, out=y)                       # packs the weights outside the capture
    want = net.infer(xb).clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        net.infer(xb, out=y)
        with torch.cuda.graph(g, stream=s):
            net.infer(xb, out=y)
    torch.cuda.current_stream().wait_stream(s)
    y.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, want)
    xb.copy_(torch.rand(4096, sur.DIMS[0], device="cuda").to(torch.bfloat16))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, net.infer(xb))
    assert sur.gemm_status() == 0
