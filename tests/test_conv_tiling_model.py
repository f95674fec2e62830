"""A CPU model of the tensor-core convolution kernels' data layout: the
padded virtual strip layout, the channel-contiguous input tile read through
shifted K-major descriptors (forward and data gradient), and the patch
matrix built from a position-contiguous tile with byte permutes (weight
gradient).  The model walks the same tiles, core matrices and descriptor
steps the kernels use, checks every shared-memory access against its buffer
and compares the result with the FP64 oracle, so that the layout argument
behind the kernels holds for ragged, strip-cut and multi-CTA cases.

The kernels' own results are compared with the oracle on the GPU
(test_gpu_surrogate.py); this file checks the scheme on any machine."""
import numpy as np
import pytest

from oracle import conv_oracle as CO

PIX, N_OUT, WT_MAX = 128, 32, 126  # positions per tile, output channels per MMA, widest strip


def _geometry(B, H, W):
    wt = W if W < WT_MAX else WT_MAX
    wv = wt + 2
    strips = (W + wt - 1) // wt
    tps = (H * wv + PIX - 1) // PIX
    return wt, wv, strips, tps, B * strips * tps


def _position(v, s, wt, wv, H, W):
    """Image (i, j) of virtual position v in strip s, or None outside the image."""
    if v < 0:
        return None
    i, jj = v // wv - 1, v % wv - 1
    j = s * wt + jj
    return (i, j) if 0 <= i < H and 0 <= j < W else None


def _read16(buf, byte, limit):
    """Eight 2-byte elements at a 16-byte aligned byte offset of a buffer."""
    assert byte % 16 == 0 and 0 <= byte and byte + 16 <= limit, (byte, limit)
    return buf[byte // 2: byte // 2 + 8]


def forward_model(x, w, bias):
    """y[b][m] = bias[m] + conv(x, w)[b][m] as the forward kernel forms it."""
    B, C, H, W = x.shape
    M = w.shape[0]
    wt, wv, strips, tps, tiles = _geometry(B, H, W)
    CH = (C + 15) // 16
    G = 2 * CH
    rows = PIX + 2 * wv + 2
    plane = rows * 16
    # weight tiles: tap t, chunk h: (t CH + h) * 1024 bytes, core matrix (rows 8a, channels 8e) at 512 e + 128 a
    sW = np.zeros(9 * CH * 512)
    for t in range(9):
        for h in range(CH):
            for m in range(M):
                for cp in range(16):
                    c = 16 * h + cp
                    if c < C:
                        byte = (t * CH + h) * 1024 + (cp // 8) * 512 + (m // 8) * 128 + (m % 8) * 16 + (cp % 8) * 2
                        sW[byte // 2] = w[m, c, t // 3, t % 3]
    y = np.full((B, M, H, W), np.nan)
    for tile in range(tiles):
        bs, k = divmod(tile, tps)
        b, s = divmod(bs, strips)
        v0 = wv + k * PIX
        vlo = v0 - wv - 1
        sX = np.zeros(G * plane // 2)
        for g in range(G):
            for r in range(rows):
                pos = _position(vlo + r, s, wt, wv, H, W)
                for q in range(8):
                    c = 8 * g + q
                    if pos is not None and c < C:
                        sX[(g * plane + r * 16) // 2 + q] = x[b, c, pos[0], pos[1]]
        D = np.zeros((PIX, N_OUT))
        for t in range(9):
            shift = (t // 3) * wv + t % 3
            for h in range(CH):
                a0 = 2 * h * plane + shift * 16  # start address; K step plane, row-group step 128
                b0 = (t * CH + h) * 1024          # K step 512, row-group step 128
                for kg in range(2):
                    A = np.stack([_read16(sX, a0 + kg * plane + (r // 8) * 128 + (r % 8) * 16, G * plane)
                                  for r in range(PIX)])
                    Bm = np.stack([_read16(sW, b0 + kg * 512 + (m // 8) * 128 + (m % 8) * 16, 9 * CH * 1024)
                                   for m in range(N_OUT)])
                    D += A @ Bm.T
        for r in range(PIX):
            v = v0 + r
            i, jj = v // wv - 1, v % wv - 1
            j = s * wt + jj
            if i < H and 0 <= jj < wt and j < W:
                assert np.isnan(y[b, 0, i, j]), "an output written twice"
                y[b, :, i, j] = D[r, :M] + bias
    return y


def weight_grad_model(x, dy):
    """dW[m][c][di][dj] = sum over pixels of dy x-patches, as the weight-gradient kernel forms it."""
    B, C, H, W = x.shape
    M = dy.shape[1]
    wt, wv, strips, tps, tiles = _geometry(B, H, W)
    Cp = 16 * ((C + 15) // 16)
    R9, RG = 9 * Cp, 9 * Cp // 8
    nblk = (R9 + 127) // 128
    xr = PIX + 2 * wv + 4
    xr += (2 - (xr & 3)) & 3
    assert xr % 4 == 2
    a_bytes, x_bytes, b_bytes = R9 * PIX * 2, Cp * xr * 2, 32 * PIX * 2
    smem = np.zeros((a_bytes + x_bytes + b_bytes) // 2)
    off_x, off_b = a_bytes, a_bytes + x_bytes
    D = np.zeros((nblk * 128, N_OUT))
    for tile in range(tiles):
        bs, k = divmod(tile, tps)
        b, s = divmod(bs, strips)
        v0 = wv + k * PIX
        vlo = v0 - wv - 1
        # input tile, position-contiguous per channel
        for c in range(Cp):
            for r in range(xr):
                pos = _position(vlo + r, s, wt, wv, H, W)
                val = x[b, c, pos[0], pos[1]] if (pos is not None and c < C) else 0.0
                smem[(off_x + (c * xr + r) * 2) // 2] = val
        # dy tile, K-major: core matrix (channels 8a, positions 8k) at 128 (4k + a); halo columns carry 0
        for m in range(32):
            for kc in range(PIX // 8):
                for e in range(8):
                    v = v0 + 8 * kc + e
                    i, jj = v // wv - 1, v % wv - 1
                    j = s * wt + jj
                    ok = m < M and i < H and 0 <= jj < wt and j < W
                    smem[(off_b + (kc * 4 + m // 8) * 128 + (m % 8) * 16) // 2 + e] = dy[b, m, i, j] if ok else 0.0
        # patch matrix rows R = t Cp + c, built from five aligned words and, for odd shifts, a byte permute
        for kc in range(PIX // 8):
            for R in range(R9):
                t, c = divmod(R, Cp)
                e0 = c * xr + (t // 3) * wv + t % 3 + 8 * kc
                w0 = e0 >> 1
                assert 2 * (w0 + 4) + 2 <= Cp * xr, "read past the input tile"
                words = [(smem[off_x // 2 + 2 * (w0 + q)], smem[off_x // 2 + 2 * (w0 + q) + 1]) for q in range(5)]
                vals = []
                for q in range(4):
                    vals += [words[q][1], words[q + 1][0]] if e0 & 1 else [words[q][0], words[q][1]]
                byte = (kc * RG + R // 8) * 128 + (R % 8) * 16
                assert byte + 16 <= a_bytes
                smem[byte // 2: byte // 2 + 8] = vals
        for blk in range(nblk):
            for kk in range(PIX // 16):
                a0, b0 = (2 * kk * RG + 16 * blk) * 128, off_b + kk * 1024
                for kg in range(2):
                    # rows of the last block past 9 Cp read the buffers that follow and are dropped
                    A = np.stack([_read16(smem, a0 + kg * RG * 128 + (r // 8) * 128 + (r % 8) * 16, smem.size * 2)
                                  for r in range(128)])
                    Bm = np.stack([_read16(smem, b0 + kg * 512 + (m // 8) * 128 + (m % 8) * 16, smem.size * 2)
                                   for m in range(N_OUT)])
                    D[blk * 128: blk * 128 + 128] += A @ Bm.T
    dw = np.zeros((M, C, 3, 3))
    for R in range(R9):
        t, c = divmod(R, Cp)
        if c < C:
            dw[:, c, t // 3, t % 3] = D[R, :M]
    return dw


FORWARD_SHAPES = [(2, 5, 32, 13, 11), (1, 3, 2, 3, 130), (2, 7, 5, 4, 3), (1, 17, 9, 5, 260), (1, 3, 2, 7, 126)]
WGRAD_SHAPES = [(2, 5, 32, 6, 11), (1, 3, 2, 3, 130), (2, 7, 5, 4, 3), (1, 17, 9, 2, 131)]


@pytest.mark.parametrize("B,C,M,H,W", FORWARD_SHAPES)
def test_forward_tiling_reproduces_the_convolution(B, C, M, H, W):
    rng = np.random.default_rng(B * 1000 + C * 100 + W)
    x = rng.uniform(-1, 1, (B, C, H, W))
    w = rng.uniform(-0.3, 0.3, (M, C, 3, 3))
    bias = rng.uniform(-0.1, 0.1, M)
    y = forward_model(x, w, bias)
    assert not np.isnan(y).any(), "an output never written"
    assert np.abs(y - CO.conv3x3(x, w, bias)).max() < 1e-12


@pytest.mark.parametrize("B,C,M,H,W", WGRAD_SHAPES)
def test_weight_gradient_tiling_reproduces_the_gradient(B, C, M, H, W):
    rng = np.random.default_rng(B * 1000 + C * 100 + W + 7)
    x = rng.uniform(-1, 1, (B, C, H, W))
    dy = rng.uniform(-1, 1, (B, M, H, W))
    _, ref, _ = CO.conv3x3_backward(x, np.zeros((M, C, 3, 3)), dy)
    assert np.abs(weight_grad_model(x, dy) - ref).max() < 1e-11
