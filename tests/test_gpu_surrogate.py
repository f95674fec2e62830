"""Learned warm start: the convolution, gradient, loss, optimiser, upsampling
and warm-start kernels (through the C ABI) against the FP64 CPU oracle, and a
short training run that fits, and what the trained network gains over the
conductive start."""
import numpy as np
import pytest

import inputs
from oracle import conv_oracle as CO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2211_03160_gb300 import tlbm

    tlbm.lib()
    return tlbm


def _bf16(a):
    import torch

    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)


def _np(t):
    import torch

    return t.float().cpu().numpy().astype(np.float64) if t.dtype == torch.bfloat16 else t.cpu().numpy().astype(np.float64)


SHAPES = [(2, 5, 32, 13, 11), (3, 32, 32, 9, 17), (1, 32, 3, 65, 65), (2, 7, 5, 4, 3), (1, 17, 9, 5, 260),
          (2, 3, 2, 3, 127)]


@pytest.mark.parametrize("B,cin,cout,H,W", SHAPES)
def test_conv_forward_backward_match_oracle(T, B, cin, cout, H, W):
    import torch

    s = torch.cuda.current_stream()
    x = _bf16(inputs.uniform_array(1 + cin, (B, cin, H, W), -1, 1)).cuda()
    w32 = torch.tensor(inputs.uniform_array(2 + cin, (cout, cin, 3, 3), -0.3, 0.3), dtype=torch.float32).cuda()
    bias = torch.tensor(inputs.uniform_array(3, (cout,), -0.1, 0.1), dtype=torch.float32).cuda()
    a = torch.empty(T.tlbm_conv3x3_weight_elems(cin), dtype=torch.bfloat16, device="cuda")
    T.tlbm_conv3x3_pack_weights(w32, cout, cin, a, s)
    w16 = w32.to(torch.bfloat16)
    y = torch.empty((B, cout, H, W), dtype=torch.float32, device="cuda")
    act = torch.empty((B, cout, H, W), dtype=torch.bfloat16, device="cuda")
    T.tlbm_conv3x3_forward(x, a, bias, y, act, B, cin, cout, H, W, 1, s)
    xr, wr = _np(x), _np(w16)
    ref = CO.conv3x3(xr, wr, _np(bias))
    scale = np.abs(ref).max()
    assert np.abs(_np(y) - ref).max() <= 1e-5 * scale
    assert np.abs(_np(act) - np.maximum(_np(y), 0)).max() <= 8e-3 * scale

    dy32 = torch.tensor(inputs.uniform_array(4, (B, cout, H, W), -1, 1), dtype=torch.float32).cuda()
    dy16 = dy32.to(torch.bfloat16)
    dyr = _np(dy16)
    rdx, rdw, rdb = CO.conv3x3_backward(xr, wr, dyr)
    dx = torch.empty((B, cin, H, W), dtype=torch.float32, device="cuda")
    at = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    T.tlbm_conv3x3_backward_data(dy16, w16, dx, B, cin, cout, H, W, at, s)
    assert np.abs(_np(dx) - rdx).max() <= 1e-5 * np.abs(rdx).max()
    ws = torch.empty(T.tlbm_conv3x3_workspace_bytes(B, cin, cout, H, W), dtype=torch.uint8, device="cuda")
    dw = torch.empty((cout, cin, 3, 3), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    T.tlbm_conv3x3_backward_weight(x, dy16, dy32, dw, db, B, cin, cout, H, W, ws, s)
    assert np.abs(_np(dw) - rdw).max() <= 1e-5 * np.abs(rdw).max()
    assert np.abs(_np(db) - _np(dy32).sum(axis=(0, 2, 3))).max() <= 1e-5 * max(1.0, np.abs(rdb).max())
    # deterministic: the same call twice gives the same bits
    dw2 = torch.empty_like(dw)
    T.tlbm_conv3x3_backward_weight(x, dy16, dy32, dw2, db, B, cin, cout, H, W, ws, s)
    assert torch.equal(dw, dw2)
    assert T.tlbm_conv3x3_status() == 0


def test_conv_training_batch_sampled_images_match_oracle(T):
    """The 32 -> 32 layer at the training batch (48 x 65 x 65 = 1585 CTAs of
    128 pixels, ragged last tile): the images are independent, so three of
    them are checked against the oracle run on that image alone."""
    import torch

    B, cin, cout, H, W = 48, 32, 32, 65, 65
    s = torch.cuda.current_stream()
    x = _bf16(inputs.uniform_array(11, (B, cin, H, W), -1, 1)).cuda()
    w32 = torch.tensor(inputs.uniform_array(12, (cout, cin, 3, 3), -0.1, 0.1), dtype=torch.float32).cuda()
    bias = torch.tensor(inputs.uniform_array(13, (cout,), -0.1, 0.1), dtype=torch.float32).cuda()
    a = torch.empty(T.tlbm_conv3x3_weight_elems(cin), dtype=torch.bfloat16, device="cuda")
    T.tlbm_conv3x3_pack_weights(w32, cout, cin, a, s)
    y = torch.empty((B, cout, H, W), dtype=torch.float32, device="cuda")
    T.tlbm_conv3x3_forward(x, a, bias, y, None, B, cin, cout, H, W, 0, s)
    dy16 = _bf16(inputs.uniform_array(14, (B, cout, H, W), -1, 1)).cuda()
    dx = torch.empty((B, cin, H, W), dtype=torch.float32, device="cuda")
    at = torch.empty(32 * 288, dtype=torch.bfloat16, device="cuda")
    w16 = w32.to(torch.bfloat16)
    T.tlbm_conv3x3_backward_data(dy16, w16, dx, B, cin, cout, H, W, at, s)
    torch.cuda.synchronize()
    assert T.tlbm_conv3x3_status() == 0
    wr, yc, dxc = _np(w16), y.cpu().numpy(), dx.cpu().numpy()
    for b in (0, 23, 47):
        xr = _np(x[b:b + 1])
        ref = CO.conv3x3(xr, wr, _np(bias))
        assert np.abs(yc[b:b + 1] - ref).max() <= 1e-5 * np.abs(ref).max()
        rdx, _, _ = CO.conv3x3_backward(xr, wr, _np(dy16[b:b + 1]))
        assert np.abs(dxc[b:b + 1] - rdx).max() <= 1e-5 * np.abs(rdx).max()


@pytest.mark.parametrize("cout,cin", [(32, 32), (3, 5), (9, 17)])
def test_packed_weight_layout(T, cout, cin):
    """The packed operand holds w[m][16h + c'][di][dj] at element
    512 (t CH + h) + 256 (c' / 8) + 64 (m / 8) + 8 (m % 8) + c' % 8, zero
    elsewhere (the documented tile order)."""
    import torch

    w32 = torch.tensor(inputs.uniform_array(31 + cin, (cout, cin, 3, 3), -1, 1), dtype=torch.float32).cuda()
    n = T.tlbm_conv3x3_weight_elems(cin)
    ch = (cin + 15) // 16
    assert n == 4608 * ch
    a = torch.full((n,), 7.0, dtype=torch.bfloat16, device="cuda")
    T.tlbm_conv3x3_pack_weights(w32, cout, cin, a, torch.cuda.current_stream())
    w16 = _np(w32.to(torch.bfloat16))
    want = np.zeros(n)
    for t in range(9):
        for h in range(ch):
            for m in range(cout):
                for cp in range(16):
                    c = 16 * h + cp
                    if c < cin:
                        want[512 * (t * ch + h) + 256 * (cp // 8) + 64 * (m // 8) + 8 * (m % 8) + cp % 8] = \
                            w16[m, c, t // 3, t % 3]
    assert np.array_equal(_np(a), want)


def test_conv_forward_with_unaligned_weight_pointer(T):
    """Weights that do not start on a 16-byte boundary take the element-wise
    staging path and give the same bits as aligned ones."""
    import torch

    B, cin, cout, H, W = 2, 7, 5, 19, 23
    s = torch.cuda.current_stream()
    n = T.tlbm_conv3x3_weight_elems(cin)
    x = _bf16(inputs.uniform_array(21, (B, cin, H, W), -1, 1)).cuda()
    w32 = torch.tensor(inputs.uniform_array(22, (cout, cin, 3, 3), -0.3, 0.3), dtype=torch.float32).cuda()
    a = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    T.tlbm_conv3x3_pack_weights(w32, cout, cin, a, s)
    store = torch.empty(n + 1, dtype=torch.bfloat16, device="cuda")
    store[1:] = a
    a_odd = store[1:]
    assert a_odd.data_ptr() % 16 != 0
    y = torch.empty((B, cout, H, W), dtype=torch.float32, device="cuda")
    y_odd = torch.empty_like(y)
    T.tlbm_conv3x3_forward(x, a, None, y, None, B, cin, cout, H, W, 0, s)
    T.tlbm_conv3x3_forward(x, a_odd, None, y_odd, None, B, cin, cout, H, W, 0, s)
    assert torch.equal(y, y_odd)
    ref = CO.conv3x3(_np(x), _np(w32.to(torch.bfloat16)), np.zeros(cout))
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_loss_relu_adam_upsample_match_oracle(T):
    import torch

    s = torch.cuda.current_stream()
    n = 3 * 65 * 65
    y = torch.tensor(inputs.uniform_array(5, (n,), -1, 1), dtype=torch.float32).cuda()
    t = torch.tensor(inputs.uniform_array(6, (n,), -1, 1), dtype=torch.float32).cuda()
    g32 = torch.empty_like(y)
    g16 = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    part = torch.zeros(1024, dtype=torch.float64, device="cuda")
    T.tlbm_mse_loss(y, t, n, g32, g16, loss, part, s)
    rl, rg = CO.mse(_np(y), _np(t))
    # the difference y - t is formed in FP32, its square summed in FP64
    assert abs(loss.item() - rl) < 1e-7 * rl and np.abs(_np(g32) - rg).max() < 1e-9

    dx = torch.tensor(inputs.uniform_array(7, (n,), -1, 1), dtype=torch.float32).cuda()
    g = torch.empty_like(dx)
    gh = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    T.tlbm_relu_backward(dx, y, n, g, gh, s)
    assert np.array_equal(_np(g), _np(dx) * (_np(y) > 0))

    w = torch.tensor(inputs.uniform_array(8, (100,), -1, 1), dtype=torch.float32).cuda()
    gr = torch.tensor(inputs.uniform_array(9, (100,), -1, 1), dtype=torch.float32).cuda()
    m = torch.zeros(100, device="cuda")
    v = torch.zeros(100, device="cuda")
    wr, mr, vr = _np(w), np.zeros(100), np.zeros(100)
    for it in (1, 2, 3):
        T.tlbm_adam_step(w, gr, m, v, 100, 1e-2, 0.9, 0.999, 1e-8, it, s)
        wr, mr, vr = CO.adam(wr, _np(gr), mr, vr, it, 1e-2)
    assert np.abs(_np(w) - wr).max() < 1e-6

    c = torch.tensor(inputs.uniform_array(10, (3, 9, 7), -1, 1), dtype=torch.float32).cuda()
    out = torch.empty((3, 65, 49), dtype=torch.float32, device="cuda")
    T.tlbm_upsample_bilinear(c, 3, 9, 7, 8, out, s)
    assert np.abs(_np(out) - CO.upsample_bilinear_vertex(_np(c), 8)).max() < 1e-6


def test_warm_start_state_matches_oracle(T, O):
    """tlbm_init_fields: f = f_eq(1, u), g = g_eq(T, u) at every node."""
    import torch

    nx, ny = 21, 17
    g = T.Sim(nx, ny, lattice=0, Ra=1e6, Pr=0.71, Ma=0.1, precision=0)
    Tf = inputs.uniform_array(11, (ny, nx), -0.5, 0.5)
    ux = inputs.uniform_array(12, (ny, nx), -0.05, 0.05)
    uy = inputs.uniform_array(13, (ny, nx), -0.05, 0.05)
    dev = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda").contiguous()
    T.tlbm_init_fields(g.h, dev(Tf), dev(ux), dev(uy), None)
    f, gg = g.get_populations()
    o = O.Sim(nx, ny, Ra=1e6, Pr=0.71, Ma=0.1)
    a_T = o.derived()["a_T"]
    e, w, _, M, Mi = O.velocity_set(0)
    T32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    for j in (0, 5, ny - 1):
        for i in (0, 7, nx - 1):
            u = [T32(ux)[j, i], T32(uy)[j, i], 0.0]
            assert np.abs(f[:, j, i] - Mi @ O.flow_meq(0, 1.0, u)).max() < 1e-15
            assert np.abs(gg[:, j, i] - O.thermal_geq(0, a_T, T32(Tf)[j, i], u)).max() < 1e-15


def test_short_training_fits(T):
    """Full-batch Adam on the project's kernels fits a smooth target field."""
    import torch

    from paper_2211_03160_gb300 import surrogate as S

    rng = np.random.default_rng(3)
    X = np.stack([S.features(10 ** rng.uniform(6, 8), rng.choice([0.71, 7.0])) for _ in range(6)])
    yy, xx = np.meshgrid(np.linspace(0, 1, 65), np.linspace(0, 1, 65), indexing="ij")
    Y = np.stack([np.stack([X[k, 0] + 0.05 * np.sin(np.pi * xx) * X[k, 3], 0.2 * np.sin(np.pi * xx) * np.sin(np.pi * yy),
                            -0.1 * np.sin(2 * np.pi * xx) * yy]) for k in range(6)]).astype(np.float32)
    net = S.ConvNet(seed=1)
    hist = S.train(net, X, Y, iters=300, lr=3e-3, log_every=100)
    assert hist[-1][1] < 0.1 * hist[0][1], hist
    pred = S.predict(net, 1e7, 0.71)
    assert pred.shape == (3, 65, 65) and torch.isfinite(pred).all()


def test_warm_start_reaches_steady_nusselt_sooner(T):
    """What the trained network gains over the conductive start.

    In a 129 x 129 cell at Pr = 0.71 and Ra between 1e4 and 3e4 the flow settles
    to one steady roll with a unique Nusselt number, so the strict criterion
    (trailing mean of Nu within 1 % of the conductive run's final value, held for
    a full free-fall time) is met by both starts.  (At Pr = 7 the conductive state
    takes longer than the run to leave.)  The network, trained on the solver's
    own time averages at other Ra, must reach that same steady state in at most
    half the conductive start's steps, for every held-out draw."""
    import torch

    from paper_2211_03160_gb300 import surrogate as S

    fine = 129
    rng = np.random.default_rng(11)
    train = [(float(10 ** rng.uniform(3.95, 4.55)), 0.71, 7000 + k) for k in range(8)]
    Y, st = S.generate(train, warm_tf=60, avg_tf=10, samples=20, fine=fine)
    assert not any(st)
    Y = S.canonical_roll(Y)
    X = np.stack([S.features(Ra, Pr, fine=fine) for Ra, Pr, _ in train])
    net = S.ConvNet(seed=0)
    hist = S.train(net, X, Y, iters=600)
    assert hist[-1][1] < 0.2 * hist[0][1]
    held_out = [(1.3e4, 0.71, 91), (1.7e4, 0.71, 92), (2.2e4, 0.71, 93)]
    ev, series = S.evaluate(net, held_out, run_tf=80, ref_tf=10, fine=fine)
    nu = np.asarray(series["nu"])
    for k, e in enumerate(ev):
        assert not e["diverged"]
        assert e["Nu_ref_rel_std"] < 1e-3, e  # steady
        final_warm = nu[len(ev) + k, -16:].mean()
        assert abs(final_warm - e["Nu_ref"]) < 0.01 * e["Nu_ref"], (e, final_warm)  # the same steady state
        assert e["held_conductive"] is not None and e["held_warm"] is not None, e
        assert e["held_warm"] <= 0.5 * e["held_conductive"], e
    torch.cuda.synchronize()
