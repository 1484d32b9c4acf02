"""tcgen05 implicit-GEMM convolutions (forward, input gradient, weight gradient) against the
FP64 CPU oracle, through the C ABI.  Inputs and weights are BF16-representable, so the only
differences are the FP32 accumulation order and the BF16 rounding of the forward output:
bound |y_gpu - y| <= 2^-8 |y| + 1e-5 sum|w||x| per element (FP32 sums, BF16 store)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import conv_ref as R  # noqa: E402


@pytest.fixture(scope="module")
def U():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import unet
    return unet


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(R.bf16_round(a), dtype=np.float32)).to(torch.bfloat16).cuda()


def tohost(t):
    return t.float().cpu().numpy().astype(np.float64)


SHAPES = [(8, 8, 8), (16, 8, 4)]
PAIRS = [(16, 16), (16, 32), (32, 64), (64, 64), (128, 64), (48, 16), (96, 32)]


@pytest.mark.parametrize("cin,cout", PAIRS)
@pytest.mark.parametrize("shape", SHAPES)
def test_conv_forward(U, cin, cout, shape):
    nz, ny, nx = shape[2], shape[1], shape[0]
    rng = np.random.default_rng(cin * 1000 + cout)
    x = R.bf16_round(rng.standard_normal((nz, ny, nx, cin)))
    w = R.bf16_round(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    for relu in (False, True):
        ref = R.conv_fwd(x, w, b.astype(np.float64), relu=relu)
        xt = bf16(x)
        wt = torch.from_numpy(w.astype(np.float32)).cuda()
        wp = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
        U.pack_weights(wt, cin, cout, 0, wp)
        y = torch.zeros((nz, ny, nx, cout), dtype=torch.bfloat16, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        U.conv3d_fwd(xt, wp, torch.from_numpy(b).cuda(), y, (nx, ny, nz), cin, cout, relu, err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        scale = R.conv_fwd(np.abs(x), np.abs(w))
        assert np.all(np.abs(tohost(y) - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)


def test_conv_forward_on_channel_slices(U):
    """Input read from channels [16, 48) of a 64-channel buffer, output written to [32, 48) of 48."""
    nx, ny, nz, cin, cout = 8, 8, 8, 32, 16
    rng = np.random.default_rng(5)
    big = R.bf16_round(rng.standard_normal((nz, ny, nx, 64)))
    w = R.bf16_round(rng.standard_normal((27, cout, cin)) / 20)
    ref = R.conv_fwd(big[..., 16:48], w)
    from paper_2501_13046_gb300.unet import Slice
    wp = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w.astype(np.float32)).cuda(), cin, cout, 0, wp)
    ybuf = torch.full((nz, ny, nx, 48), 7.0, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    U.conv3d_fwd(Slice(bf16(big), 16, 32), wp, None, Slice(ybuf, 32, 16), (nx, ny, nz), cin, cout, False, err)
    torch.cuda.synchronize()
    out = tohost(ybuf)
    assert np.all(out[..., :32] == 7.0)   # outside the slice untouched
    scale = R.conv_fwd(np.abs(big[..., 16:48]), np.abs(w))
    assert np.all(np.abs(out[..., 32:48] - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 48), (32, 96), (64, 64)])
def test_conv_input_gradient(U, cin, cout):
    """dX = conv of dY with flipped, transposed weights (packing mode 1), forward kernel."""
    nx, ny, nz = 8, 8, 8
    rng = np.random.default_rng(11)
    dy = R.bf16_round(rng.standard_normal((nz, ny, nx, cout)))
    w = R.bf16_round(rng.standard_normal((27, cout, cin)) / 10)
    ref = R.conv_dgrad(dy, w)
    wp = torch.empty((27, cin, cout), dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w.astype(np.float32)).cuda(), cin, cout, 1, wp)
    dx = torch.zeros((nz, ny, nx, cin), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    U.conv3d_fwd(bf16(dy), wp, None, dx, (nx, ny, nz), cout, cin, False, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale = R.conv_dgrad(np.abs(dy), np.abs(w))
    assert np.all(np.abs(tohost(dx) - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)


@pytest.mark.parametrize("cin,cout", [(16, 16), (16, 32), (48, 16), (64, 64), (128, 64), (96, 32)])
def test_conv_weight_gradient(U, cin, cout):
    nx, ny, nz = 16, 8, 8
    rng = np.random.default_rng(21)
    x = R.bf16_round(rng.standard_normal((nz, ny, nx, cin)))
    dy = R.bf16_round(rng.standard_normal((nz, ny, nx, cout)))
    ref = R.conv_wgrad(x, dy)
    dw = torch.zeros((27, cout, cin), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    U.conv3d_wgrad(bf16(x), bf16(dy), dw, (nx, ny, nz), cin, cout, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale = R.conv_wgrad(np.abs(x), np.abs(dy))   # FP32 accumulation over 1024 voxels
    np.testing.assert_array_less(np.abs(dw.cpu().numpy() - ref), 1e-5 * scale + 1e-6)


BLOCK_SHAPES = [(16, 16, 4), (8, 32, 6)]   # nx % 8 == 0, ny % 16 == 0, nz even: the block-tile kernel
BLOCK_PAIRS = [(16, 16), (16, 32), (16, 48), (32, 16), (32, 32), (32, 64), (48, 16)]


@pytest.mark.parametrize("cin,cout", BLOCK_PAIRS)
@pytest.mark.parametrize("shape", BLOCK_SHAPES)
def test_conv_forward_block_tiles(U, cin, cout, shape):
    """Volumes the block-tile kernel takes (8 x 16 x 2 voxel tiles, input block and all weights in
    shared memory, shifted descriptors per tap), against the FP64 oracle with the same bound."""
    nz, ny, nx = shape[2], shape[1], shape[0]
    rng = np.random.default_rng(cin * 977 + cout + nx)
    x = R.bf16_round(rng.standard_normal((nz, ny, nx, cin)))
    w = R.bf16_round(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    wp = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w.astype(np.float32)).cuda(), cin, cout, 0, wp)
    for relu in (False, True):
        ref = R.conv_fwd(x, w, b.astype(np.float64), relu=relu)
        y = torch.zeros((nz, ny, nx, cout), dtype=torch.bfloat16, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        U.conv3d_fwd(bf16(x), wp, torch.from_numpy(b).cuda(), y, (nx, ny, nz), cin, cout, relu, err)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        scale = R.conv_fwd(np.abs(x), np.abs(w))
        assert np.all(np.abs(tohost(y) - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)


def test_conv_block_tiles_on_channel_slices_and_input_gradient(U):
    """Block-tile kernel reading channels [16, 64) of a 64-channel buffer into channels [16, 32) of
    a 32-channel one, and the input gradient (flipped, transposed weights) of a (16 -> 48) layer."""
    nx, ny, nz = 16, 16, 4
    rng = np.random.default_rng(21)
    big = R.bf16_round(rng.standard_normal((nz, ny, nx, 64)))
    w = R.bf16_round(rng.standard_normal((27, 16, 48)) / 30)
    ref = R.conv_fwd(big[..., 16:64], w)
    from paper_2501_13046_gb300.unet import Slice
    wp = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w.astype(np.float32)).cuda(), 48, 16, 0, wp)
    ybuf = torch.full((nz, ny, nx, 32), 7.0, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    U.conv3d_fwd(Slice(bf16(big), 16, 48), wp, None, Slice(ybuf, 16, 16), (nx, ny, nz), 48, 16, False, err)
    torch.cuda.synchronize()
    out = tohost(ybuf)
    assert np.all(out[..., :16] == 7.0)
    scale = R.conv_fwd(np.abs(big[..., 16:64]), np.abs(w))
    assert np.all(np.abs(out[..., 16:32] - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)
    # input gradient of a 16 -> 48 convolution: the forward kernel with 48 -> 16 packed weights
    dy = R.bf16_round(rng.standard_normal((nz, ny, nx, 48)))
    w2 = R.bf16_round(rng.standard_normal((27, 48, 16)) / 10)
    ref2 = R.conv_dgrad(dy, w2)
    wp2 = torch.empty((27, 16, 48), dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w2.astype(np.float32)).cuda(), 16, 48, 1, wp2)
    dx = torch.zeros((nz, ny, nx, 16), dtype=torch.bfloat16, device="cuda")
    U.conv3d_fwd(bf16(dy), wp2, None, dx, (nx, ny, nz), 48, 16, False, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale2 = R.conv_dgrad(np.abs(dy), np.abs(w2))
    assert np.all(np.abs(tohost(dx) - ref2) <= 2 ** -8 * np.abs(ref2) + 1e-5 * scale2 + 1e-6)


# 4, 4, 32 and 128 tiles: 27, 27, 14 and 5 groups (ny = 8: never the block-tile kernel)
SPLIT_SHAPES = [(8, 8, 8), (16, 8, 4), (16, 8, 32), (32, 8, 64)]


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 64), (64, 64), (128, 64), (96, 32), (48, 16)])
@pytest.mark.parametrize("shape", SPLIT_SHAPES)
def test_conv_forward_split_taps(U, cin, cout, shape):
    """The split-K form (taps in groups of CTAs, FP32 partials added in group order): the same bound
    against the FP64 oracle, bitwise repeatable, and a workspace below the query is rejected."""
    nz, ny, nx = shape[2], shape[1], shape[0]
    rng = np.random.default_rng(cin * 31 + cout * 7 + nx * ny * nz)
    x = R.bf16_round(rng.standard_normal((nz, ny, nx, cin)))
    w = R.bf16_round(rng.standard_normal((27, cout, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    wp = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w.astype(np.float32)).cuda(), cin, cout, 0, wp)
    wsb = U.conv3d_workspace((nx, ny, nz), cout)
    assert wsb > 0
    ws = torch.full((wsb // 4,), float("nan"), dtype=torch.float32, device="cuda")
    xt, bt = bf16(x), torch.from_numpy(b).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for relu in (False, True):
        ref = R.conv_fwd(x, w, b.astype(np.float64), relu=relu)
        ys = []
        for _ in range(2):
            y = torch.zeros((nz, ny, nx, cout), dtype=torch.bfloat16, device="cuda")
            U.conv3d_fwd(xt, wp, bt, y, (nx, ny, nz), cin, cout, relu, err, ws=ws)
            ys.append(y)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(ys[0], ys[1])
        scale = R.conv_fwd(np.abs(x), np.abs(w))
        assert np.all(np.abs(tohost(ys[0]) - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)
    with pytest.raises(RuntimeError):
        U.conv3d_fwd(xt, wp, bt, ys[0], (nx, ny, nz), cin, cout, False, err, ws=ws[: wsb // 4 - 4])


def test_conv_split_taps_on_channel_slices_and_input_gradient(U):
    """Split-K form on channel slices (input [16, 48) of 64, output [32, 48) of 48; the rest
    untouched) and as the input gradient of a (32 -> 96) layer on a 16 x 8 x 32 grid."""
    from paper_2501_13046_gb300.unet import Slice
    nx, ny, nz, cin, cout = 16, 8, 32, 32, 16
    rng = np.random.default_rng(55)
    big = R.bf16_round(rng.standard_normal((nz, ny, nx, 64)))
    w = R.bf16_round(rng.standard_normal((27, cout, cin)) / 20)
    ref = R.conv_fwd(big[..., 16:48], w)
    wp = torch.empty(w.shape, dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w.astype(np.float32)).cuda(), cin, cout, 0, wp)
    ws = torch.empty(U.conv3d_workspace((nx, ny, nz), 96) // 4, dtype=torch.float32, device="cuda")
    ybuf = torch.full((nz, ny, nx, 48), 7.0, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    U.conv3d_fwd(Slice(bf16(big), 16, 32), wp, None, Slice(ybuf, 32, 16), (nx, ny, nz), cin, cout, False, err,
                 ws=ws)
    torch.cuda.synchronize()
    out = tohost(ybuf)
    assert np.all(out[..., :32] == 7.0)
    scale = R.conv_fwd(np.abs(big[..., 16:48]), np.abs(w))
    assert np.all(np.abs(out[..., 32:48] - ref) <= 2 ** -8 * np.abs(ref) + 1e-5 * scale + 1e-6)
    dy = R.bf16_round(rng.standard_normal((nz, ny, nx, 96)))
    w2 = R.bf16_round(rng.standard_normal((27, 96, 32)) / 10)
    ref2 = R.conv_dgrad(dy, w2)
    wp2 = torch.empty((27, 32, 96), dtype=torch.bfloat16, device="cuda")
    U.pack_weights(torch.from_numpy(w2.astype(np.float32)).cuda(), 32, 96, 1, wp2)
    dx = torch.zeros((nz, ny, nx, 32), dtype=torch.bfloat16, device="cuda")
    U.conv3d_fwd(bf16(dy), wp2, None, dx, (nx, ny, nz), 96, 32, False, err, ws=ws)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale2 = R.conv_dgrad(np.abs(dy), np.abs(w2))
    assert np.all(np.abs(tohost(dx) - ref2) <= 2 ** -8 * np.abs(ref2) + 1e-5 * scale2 + 1e-6)
