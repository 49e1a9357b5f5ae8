"""The learned start's network on the GPU against the FP64 oracle (oracle/fno.py):
forward values, gradients (central finite differences of the oracle), training."""
import numpy as np
import pytest

from oracle import fno as OF

pytestmark = pytest.mark.gpu

N, M, WID, LAY, CIN, COUT, B = 12, 3, 8, 2, 7, 6, 2


@pytest.fixture(scope="module")
def fh():
    import torch
    assert torch.cuda.is_available()
    from paper_1701_04685_gb300 import build
    build.build()
    import paper_1701_04685_gb300 as fh
    return fh


def bf16(a):
    """Round float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def random_params(rng):
    p = OF.Params(CIN, COUT, WID, M, LAY)
    p.P = rng.standard_normal(p.P.shape) / np.sqrt(CIN)
    p.p = 0.1 * rng.standard_normal(p.p.shape)
    p.W = bf16(rng.standard_normal(p.W.shape) / np.sqrt(WID))
    p.w = 0.1 * rng.standard_normal(p.w.shape)
    s = 1.0 / WID
    p.R = bf16(s * rng.standard_normal(p.R.shape)) + 1j * bf16(s * rng.standard_normal(p.R.shape))
    p.Q = rng.standard_normal(p.Q.shape) / np.sqrt(WID)
    p.q = 0.1 * rng.standard_normal(p.q.shape)
    # the product stores FP32 master weights: make every parameter FP32-exact
    p.set_flat(p.flat().astype(np.float32).astype(np.float64))
    return p


def _net(fh, p):
    net = fh.FNO(N, CIN, COUT, WID, M, LAY, max_batch=B)
    net.set_params(p.flat().astype(np.float32))
    return net


def test_param_round_trip(fh, rng):
    p = random_params(rng)
    net = _net(fh, p)
    assert np.array_equal(net.get_params().astype(np.float64), p.flat())


def test_forward_matches_oracle(fh, rng):
    import torch
    p = random_params(rng)
    net = _net(fh, p)
    x = rng.standard_normal((B, CIN, N, N, N)).astype(np.float32)
    y = torch.empty((B, COUT, N ** 3), dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(x.reshape(B, CIN, -1)).cuda(), y)
    got = y.cpu().numpy().reshape(B, COUT, N, N, N)
    for b in range(B):
        ref = OF.forward(p, x[b].astype(np.float64))
        assert np.abs(got[b] - ref).max() / np.abs(ref).max() < 2e-5


def test_gradients_match_oracle_finite_differences(fh, rng):
    import torch
    p = random_params(rng)
    net = _net(fh, p)
    x = rng.standard_normal((B, CIN, N, N, N)).astype(np.float32)
    t = rng.standard_normal((B, COUT, N, N, N)).astype(np.float32)
    net.zero_grad()
    loss = net.loss_grad(torch.from_numpy(x.reshape(B, CIN, -1)).cuda(), torch.from_numpy(t.reshape(B, COUT, -1)).cuda())
    xs = [x[b].astype(np.float64) for b in range(B)]
    ts = [t[b].astype(np.float64) for b in range(B)]
    assert abs(loss - OF.loss(p, xs, ts)) / OF.loss(p, xs, ts) < 1e-5
    g = net.get_grads().astype(np.float64)
    theta = p.flat()
    sizes = [p.P.size, p.p.size, p.W.size, p.w.size, p.R.size, p.R.size, p.Q.size, p.q.size]
    names = ["P", "p", "W", "w", "ReR", "ImR", "Q", "q"]
    o = 0
    q = OF.Params(CIN, COUT, WID, M, LAY)
    for name, n in zip(names, sizes):
        d = np.zeros_like(theta)
        d[o:o + n] = rng.standard_normal(n)
        h = 1e-4 / np.abs(d).max()
        q.set_flat(theta + h * d)
        lp = OF.loss(q, xs, ts)
        q.set_flat(theta - h * d)
        lm = OF.loss(q, xs, ts)
        fd = (lp - lm) / (2 * h)
        an = float(g @ d)
        assert abs(fd - an) <= 2e-3 * abs(fd) + 1e-9, (name, fd, an)
        o += n


def test_training_reduces_the_loss(fh, rng):
    import torch
    p = random_params(rng)
    net = _net(fh, p)
    x = torch.from_numpy(rng.standard_normal((B, CIN, N ** 3)).astype(np.float32)).cuda()
    t = torch.from_numpy(0.3 * rng.standard_normal((B, COUT, N ** 3)).astype(np.float32)).cuda()
    first = None
    for step in range(1, 151):
        net.zero_grad()
        loss = net.loss_grad(x, t)
        first = loss if first is None else first
        net.adam_step(3e-3, step)
    assert loss < 0.5 * first


def test_make_input_channels(fh):
    import torch
    net = fh.FNO(8, CIN, COUT, 4, 2, 1, max_batch=1)
    phase = torch.tensor(np.arange(512) % 2, dtype=torch.uint8, device="cuda")
    x = torch.empty((CIN, 512), dtype=torch.float32, device="cuda")
    e0 = np.array([0.1, -0.2, 0.3, 0.4, 0.5, 0.6])
    net.make_input(phase, [0.0, 2.0], e0, x)
    xc = x.cpu().numpy()
    assert np.allclose(xc[0], np.where(np.arange(512) % 2 == 1, 1.0, 0.0))
    for c in range(6):
        assert np.allclose(xc[c + 1], e0[c])


def _params(rng, cin, cout, width, modes, layers):
    p = OF.Params(cin, cout, width, modes, layers)
    p.P = rng.standard_normal(p.P.shape) / np.sqrt(cin)
    p.p = 0.1 * rng.standard_normal(p.p.shape)
    p.W = bf16(rng.standard_normal(p.W.shape) / np.sqrt(width))
    p.w = 0.1 * rng.standard_normal(p.w.shape)
    s = 1.0 / width
    p.R = bf16(s * rng.standard_normal(p.R.shape)) + 1j * bf16(s * rng.standard_normal(p.R.shape))
    p.Q = rng.standard_normal(p.Q.shape) / np.sqrt(width)
    p.q = 0.1 * rng.standard_normal(p.q.shape)
    p.set_flat(p.flat().astype(np.float32).astype(np.float64))
    return p


@pytest.mark.parametrize("n,width", [(16, 16), (16, 32), (32, 32)])
def test_tensor_core_layers_match_simt_layers_and_oracle(fh, n, width):
    """The hidden 1 x 1 layers on tcgen05 (split-BF16 activations, FP32
    accumulation in tensor memory) against the SIMT layers and the FP64 network
    oracle, forward and loss."""
    import torch
    rng = np.random.default_rng(21 + n + width)
    p = _params(rng, 1, 6, width, 4, 2)
    net = fh.FNO(n, 1, 6, width, 4, 2, max_batch=2)
    net.set_params(p.flat().astype(np.float32))
    xs = rng.standard_normal((2, 1, n, n, n)).astype(np.float32)
    x = torch.from_numpy(xs.reshape(2, 1, -1)).cuda()
    y_tc = torch.empty((2, 6, n ** 3), dtype=torch.float32, device="cuda")
    y_simt = torch.empty_like(y_tc)
    net.set_tensor_cores(True)
    net.forward(x, y_tc)
    t = torch.zeros_like(y_tc)
    l_tc = net.loss_grad(x, t)
    net.set_tensor_cores(False)
    net.forward(x, y_simt)
    l_simt = net.loss_grad(x, t)
    a, b = y_tc.cpu().numpy(), y_simt.cpu().numpy()
    assert np.abs(a - b).max() / np.abs(b).max() < 2e-6
    assert abs(l_tc - l_simt) / l_simt < 1e-5
    for k in range(2):
        ref = OF.forward(p, xs[k].astype(np.float64)).reshape(6, -1)
        assert np.abs(a[k] - ref).max() / np.abs(ref).max() < 2e-5
    net.close()
