"""Latent bitstream: fixed-point ARM, Laplace frequency tables, range coder -- TEST
INFRASTRUCTURE ONLY.

Same import rule as ``oracle.coolchic``: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module; the product path runs the CUDA library.

What it restates.  Sec. II "Encoding": once the encoder has converged, the latents are
entropy coded with a range coder driven by the ARM's probability model p_psi; Sec. II
"Decoding" (items i-iii, Fig. 2): the decoder reads the latent grids with that model,
level by level, each latent conditioned on its already-decoded causal neighbours, then
upsamples and synthesises the image.  The decoder re-evaluates the ARM on decoded values,
so encoder and decoder must agree on every probability to the last bit; the paper does
not say how (its C decoder is Sec. III-B "Fast C implementation").  Readings taken here,
all of them integer-exact so that two implementations agree bit for bit:

* ARM in 32-bit fixed point with 8 fractional bits (Q8).  Weights are rounded (half to
  even) to multiples of 2^-8 and clamped to +-2^11 in Q8 units (|w| <= 8), biases to
  +-2^15 (|b| <= 128).  The context values are the integer latents clamped to [-128, 128]
  times 256.  A layer computes z = ((sum_j W[o, j] a[j]) + 128) >> 8 + b[o] (arithmetic
  shift, i.e. round half up of the Q16 sum), saturated to +-2^15; a LinR layer outputs
  a[o] + max(z, 0), saturated to +-2^15; the output layer gives (mu_q, s_q) in Q8.  With
  N <= 24 every sum is below 24 * 2^11 * 2^15 < 2^31: the whole ARM is exact in int32.
* Probability tables.  The log-scale s_q selects one of NSCALE bins of width 1/8 starting
  at LOGB_LO_Q / 256 (= floor(256 ln 0.01) / 256), clamped to the first and last bin;
  mu_q splits into m = floor(mu_q / 256) and one of NMU = 8 fractional bins.  Table
  (bin j, fraction fi) is the Laplace law of mean (fi + 1/2) / 8 and scale
  exp(LOGB_LO_Q / 256 + (j + 1/2) / 8) over the symbols k = y_hat - m in [-A, A], plus
  one escape symbol for each tail (k < -A, k > A), whose masses are the tail masses.
  Each of the NSYM = 2A + 3 masses p becomes the frequency 1 + floor(p (2^16 - NSYM));
  what is left of 2^16 goes to the first symbol of largest frequency.  All table
  arithmetic is IEEE double with the C library's exp.
* Escaped symbols: the excess e = |k| - A - 1 follows as an order-0 Exp-Golomb code of
  e + 1 in equiprobable binary decisions.
* Range coder: 32-bit range, 33-bit low with carry propagation through a pending 0xFF
  run, byte output, frequencies out of 2^16.  The always-zero first byte is not written;
  the final value is the one of the last interval with the most trailing zero bits, and
  trailing zero bytes are not written (a decoder reads zeros past the end).
* Substreams: one per latent row (level-major, rows top to bottom), so that a decoder
  may run the rows as a wavefront: row r may decode position x once row r - 1 has
  passed x + lag - 1, with lag = max over context offsets (dy < 0, dx) of
  ceil((dx + 1) / -dy).
* Bitstream: magic b"CCF1", H and W (u32 LE), the 7 architecture bytes and a zero pad,
  the fixed-point ARM parameters (i32 LE, flat parameter order), the upsampling and
  synthesis parameters (f32 LE, flat parameter order), the byte count of every
  substream (LEB128), the substreams.
"""
from __future__ import annotations

import bisect
import math
import struct

import numpy as np

from .coolchic import Arch, causal_offsets, param_shapes

Q_FRAC = 8
W_LIM = 1 << 11
ACT_LIM = 1 << 15
CTX_LIM = 128
Y_LIM = 1 << 20
PROB_BITS = 16
TOTAL = 1 << PROB_BITS
A = 64
NSYM = 2 * A + 3
NMU = 8
LOGB_LO_Q = math.floor(256.0 * math.log(1e-2))   # -1179
LOGB_STEP_Q = 32                                   # 1/8 in Q8
NSCALE = 93                                        # bins reach past ln 1e3
MAGIC = b"CCF1"


# --------------------------------------------------------------------------------------
# Fixed-point ARM
# --------------------------------------------------------------------------------------

def arm_param_names(arch: Arch):
    return [n for n, _ in param_shapes(arch) if n.startswith("arm.")]


def quantize_arm(named: dict, arch: Arch) -> dict:
    """Q8 integers of the ARM weights (clamped to +-W_LIM) and biases (+-ACT_LIM)."""
    out = {}
    for name in arm_param_names(arch):
        v = np.rint(np.asarray(named[name], np.float64) * (1 << Q_FRAC)).astype(np.int64)
        lim = W_LIM if ".w" in name else ACT_LIM
        out[name] = np.clip(v, -lim, lim)
    return out


def _sat(v):
    return np.clip(v, -ACT_LIM, ACT_LIM)


def _layer(a, W, b):
    """((a W^T) + 128) >> 8 + b; the sum is checked to fit int32, as the format promises."""
    acc = a @ W.T
    assert np.abs(acc).max(initial=0) < 2 ** 31 - (1 << (Q_FRAC - 1))
    return ((acc + (1 << (Q_FRAC - 1))) >> Q_FRAC) + b


def arm_fixed(ctx_int: np.ndarray, Q: dict, arch: Arch):
    """[..., N] integer contexts -> (mu_q, s_q) in Q8 (int64 arrays holding int32 values)."""
    a = np.clip(np.asarray(ctx_int, np.int64), -CTX_LIM, CTX_LIM) << Q_FRAC
    for i in range(arch.arm_layers):
        z = _sat(_layer(a, Q[f"arm.w{i}"], Q[f"arm.b{i}"]))
        a = _sat(a + np.maximum(z, 0))
    out = _sat(_layer(a, Q["arm.wout"], Q["arm.bout"]))
    return out[..., 0], out[..., 1]


def context_int(plane: np.ndarray, offsets) -> np.ndarray:
    """[h, w] integer plane -> [h, w, N] causal contexts, 0 outside the grid."""
    h, w = plane.shape
    r = max(max(-dy, abs(dx)) for dy, dx in offsets)
    p = np.zeros((h + r, w + 2 * r), np.int64)
    p[r:, r:r + w] = plane
    return np.stack([p[r + dy:r + dy + h, r + dx:r + dx + w] for dy, dx in offsets], -1)


def wavefront_lag(offsets) -> int:
    return max(-(-(dx + 1) // -dy) for dy, dx in offsets if dy < 0)


# --------------------------------------------------------------------------------------
# Probability tables
# --------------------------------------------------------------------------------------

def table_index(mu_q, s_q):
    """(table number j * NMU + fi, integer part m of mu) for Q8 ARM outputs."""
    mu_q = np.asarray(mu_q, np.int64)
    s_q = np.asarray(s_q, np.int64)
    j = np.clip((s_q - LOGB_LO_Q) >> 5, 0, NSCALE - 1)
    fi = (mu_q & 255) >> 5
    return j * NMU + fi, mu_q >> Q_FRAC


def laplace_freqs(j: int, fi: int):
    """The NSYM frequencies of table (j, fi); they sum to TOTAL and are all >= 1."""
    b = math.exp(LOGB_LO_Q / 256.0 + (j + 0.5) / 8.0)
    f = (fi + 0.5) / NMU

    def F(x):
        z = (x - f) / b
        return 0.5 * math.exp(z) if z < 0.0 else 1.0 - 0.5 * math.exp(-z)

    masses = [F(-A - 0.5)]
    masses += [F(k + 0.5) - F(k - 0.5) for k in range(-A, A + 1)]
    masses.append(1.0 - F(A + 0.5))
    freq = [1 + math.floor(p * (TOTAL - NSYM)) for p in masses]
    rest = TOTAL - sum(freq)
    assert rest >= 0
    top = max(freq)
    freq[freq.index(top)] += rest
    return freq


def build_tables() -> np.ndarray:
    """[NSCALE * NMU, NSYM + 1] cumulative frequencies (first column 0, last TOTAL)."""
    cum = np.zeros((NSCALE * NMU, NSYM + 1), np.int64)
    for j in range(NSCALE):
        for fi in range(NMU):
            cum[j * NMU + fi, 1:] = np.cumsum(laplace_freqs(j, fi))
    return cum


# --------------------------------------------------------------------------------------
# Range coder
# --------------------------------------------------------------------------------------

class RangeEncoder:
    def __init__(self):
        self.low = 0              # up to 33 bits: bit 32 is a carry into the pending bytes
        self.range = 0xFFFFFFFF
        self.cache = 0            # last byte held back (a carry may still reach it)
        self.pending = 1          # cache byte + number of 0xFF bytes behind it
        self.first = True         # the first cache byte is always 0 and is not written
        self.out = bytearray()

    def _shift_low(self):
        if self.low < 0xFF000000 or self.low >= 1 << 32:
            carry = self.low >> 32
            if self.first:
                assert self.cache + carry == 0
                self.first = False
            else:
                self.out.append((self.cache + carry) & 0xFF)
            for _ in range(self.pending - 1):
                self.out.append((0xFF + carry) & 0xFF)
            self.pending = 0
            self.cache = (self.low >> 24) & 0xFF
        self.pending += 1
        self.low = (self.low & 0x00FFFFFF) << 8

    def encode(self, start: int, freq: int):
        """Code the interval [start, start + freq) out of TOTAL."""
        r = self.range >> PROB_BITS
        self.low += r * start
        self.range = r * freq
        while self.range < 1 << 24:
            self.range <<= 8
            self._shift_low()

    def encode_bit(self, bit: int):
        self.encode(bit << (PROB_BITS - 1), 1 << (PROB_BITS - 1))

    def finish(self) -> bytes:
        """Flush with the value of [low, low + range) that has the most trailing zero
        bits, then drop trailing zero bytes: a decoder reads zeros past the end."""
        top = self.low + self.range - 1
        for k in range(32, -1, -1):
            v = top & ~((1 << k) - 1)
            if v >= self.low:
                break
        self.low = v
        for _ in range(5):
            self._shift_low()
        while self.out and self.out[-1] == 0:
            self.out.pop()
        return bytes(self.out)


class RangeDecoder:
    def __init__(self, data: bytes):
        self.data = data
        self.pos = 0
        self.range = 0xFFFFFFFF
        self.code = 0
        self.r = 0
        for _ in range(4):
            self.code = (self.code << 8) | self._byte()

    def _byte(self) -> int:
        b = self.data[self.pos] if self.pos < len(self.data) else 0
        self.pos += 1
        return b

    def target(self) -> int:
        """The frequency value the next symbol's interval contains."""
        self.r = self.range >> PROB_BITS
        return min(self.code // self.r, TOTAL - 1)

    def consume(self, start: int, freq: int):
        self.code -= self.r * start
        self.range = self.r * freq
        while self.range < 1 << 24:
            self.code = (self.code << 8) | self._byte()
            self.range <<= 8

    def decode_bit(self) -> int:
        bit = 1 if self.target() >= 1 << (PROB_BITS - 1) else 0
        self.consume(bit << (PROB_BITS - 1), 1 << (PROB_BITS - 1))
        return bit


def _encode_excess(enc: RangeEncoder, e: int):
    v = e + 1
    n = v.bit_length() - 1
    for _ in range(n):
        enc.encode_bit(1)
    enc.encode_bit(0)
    for i in range(n - 1, -1, -1):
        enc.encode_bit((v >> i) & 1)


def _decode_excess(dec: RangeDecoder) -> int:
    n = 0
    while dec.decode_bit():
        n += 1
    v = 1
    for _ in range(n):
        v = (v << 1) | dec.decode_bit()
    return v - 1


def encode_symbol(enc: RangeEncoder, cum_row, k: int):
    """Code k = y_hat - m with the table row cum_row."""
    if k < -A:
        idx = 0
    elif k > A:
        idx = NSYM - 1
    else:
        idx = k + A + 1
    enc.encode(int(cum_row[idx]), int(cum_row[idx + 1] - cum_row[idx]))
    if idx == 0:
        _encode_excess(enc, -A - 1 - k)
    elif idx == NSYM - 1:
        _encode_excess(enc, k - A - 1)


def decode_symbol(dec: RangeDecoder, cum_row) -> int:
    t = dec.target()
    idx = bisect.bisect_right(cum_row, t) - 1
    dec.consume(int(cum_row[idx]), int(cum_row[idx + 1] - cum_row[idx]))
    if idx == 0:
        return -A - 1 - _decode_excess(dec)
    if idx == NSYM - 1:
        return A + 1 + _decode_excess(dec)
    return idx - A - 1


# --------------------------------------------------------------------------------------
# Substreams and bitstream
# --------------------------------------------------------------------------------------

def row_context(plane: np.ndarray, r: int, offsets) -> np.ndarray:
    """[w, N] causal contexts of row r (only the rows the offsets reach are read)."""
    r0 = max(0, r - max(-dy for dy, _ in offsets))
    return context_int(plane[r0:r + 1], offsets)[r - r0]


def encode_rows(plane: np.ndarray, Q: dict, arch: Arch, cum: np.ndarray, rows=None):
    """Substreams (bytes) of the given rows (default: all) of one level's integer plane."""
    offs = causal_offsets(arch.arm_ctx)
    out = []
    for r in (range(plane.shape[0]) if rows is None else rows):
        mu_q, s_q = arm_fixed(row_context(plane, r, offs), Q, arch)
        t, m = table_index(mu_q, s_q)
        enc = RangeEncoder()
        for x in range(plane.shape[1]):
            encode_symbol(enc, cum[t[x]], int(plane[r, x]) - int(m[x]))
        out.append(enc.finish())
    return out


def decode_level(streams, h: int, w: int, Q: dict, arch: Arch, cum: np.ndarray):
    """Rows in raster order, each latent from its decoded causal context."""
    offs = causal_offsets(arch.arm_ctx)
    plane = np.zeros((h, w), np.int64)
    for r in range(h):
        dec = RangeDecoder(streams[r])
        for x in range(w):
            c = [int(plane[r + dy, x + dx]) if 0 <= r + dy and 0 <= x + dx < w else 0
                 for dy, dx in offs]
            mu_q, s_q = arm_fixed(np.array(c, np.int64), Q, arch)
            t, m = table_index(mu_q, s_q)
            plane[r, x] = int(m) + decode_symbol(dec, cum[int(t)])
    return plane


def _leb128(n: int) -> bytes:
    out = bytearray()
    while True:
        b = n & 0x7F
        n >>= 7
        out.append(b | (0x80 if n else 0))
        if not n:
            return bytes(out)


def _read_leb128(buf: bytes, pos: int):
    n, shift = 0, 0
    while True:
        b = buf[pos]
        pos += 1
        n |= (b & 0x7F) << shift
        shift += 7
        if not b & 0x80:
            return n, pos


def arch_bytes(arch: Arch) -> bytes:
    return bytes([arch.levels, arch.arm_ctx, arch.arm_layers, arch.up_kernel,
                  int(arch.up_per_level), arch.syn_hidden, arch.syn_res3x3, 0])


def write_bitstream(H: int, W: int, arch: Arch, named: dict, y_levels) -> bytes:
    """The whole bitstream for integer latents y_levels and float32 parameters named."""
    Q = quantize_arm(named, arch)
    cum = build_tables()
    for y in y_levels:
        assert np.abs(np.asarray(y, np.int64)).max(initial=0) <= Y_LIM
    out = bytearray(MAGIC + struct.pack("<II", H, W) + arch_bytes(arch))
    for name in arm_param_names(arch):
        out += np.asarray(Q[name], "<i4").tobytes()
    for name, _ in param_shapes(arch):
        if not name.startswith("arm."):
            out += np.asarray(named[name], "<f4").tobytes()
    streams = []
    for y in y_levels:
        streams += encode_rows(np.asarray(y, np.int64), Q, arch, cum)
    for s in streams:
        out += _leb128(len(s))
    for s in streams:
        out += s
    return bytes(out)


def read_bitstream(bs: bytes):
    """-> (H, W, arch, float parameters by name (ARM: Q8 / 256), integer latent levels)."""
    assert bs[:4] == MAGIC
    H, W = struct.unpack_from("<II", bs, 4)
    ab = bs[12:20]
    arch = Arch(levels=ab[0], arm_ctx=ab[1], arm_layers=ab[2], up_kernel=ab[3],
                up_per_level=bool(ab[4]), syn_hidden=ab[5], syn_res3x3=ab[6])
    pos = 20
    Q, named = {}, {}
    for name, shape in param_shapes(arch):
        n = int(np.prod(shape))
        if name.startswith("arm."):
            Q[name] = np.frombuffer(bs, "<i4", n, pos).astype(np.int64).reshape(shape)
            named[name] = Q[name] / float(1 << Q_FRAC)
        else:
            named[name] = np.frombuffer(bs, "<f4", n, pos).astype(np.float32).reshape(shape)
        pos += 4 * n
    shapes = [(-(-H // (1 << l)), -(-W // (1 << l))) for l in range(arch.levels)]
    lens = []
    for h, _ in shapes:
        for _ in range(h):
            n, pos = _read_leb128(bs, pos)
            lens.append(n)
    streams = []
    for n in lens:
        streams.append(bs[pos:pos + n])
        pos += n
    cum = build_tables()
    levels, k = [], 0
    for h, w in shapes:
        levels.append(decode_level(streams[k:k + h], h, w, Q, arch, cum))
        k += h
    return H, W, arch, named, levels


def header_and_streams(bs: bytes):
    """(byte offset where the substream lengths start, [substream bytes]) of a bitstream."""
    H, W = struct.unpack_from("<II", bs, 4)
    ab = bs[12:20]
    arch = Arch(levels=ab[0], arm_ctx=ab[1], arm_layers=ab[2], up_kernel=ab[3],
                up_per_level=bool(ab[4]), syn_hidden=ab[5], syn_res3x3=ab[6])
    pos = 20 + 4 * sum(int(np.prod(s)) for _, s in param_shapes(arch))
    start = pos
    rows = sum(-(-H // (1 << l)) for l in range(arch.levels))
    lens = []
    for _ in range(rows):
        n, pos = _read_leb128(bs, pos)
        lens.append(n)
    streams = []
    for n in lens:
        streams.append(bs[pos:pos + n])
        pos += n
    assert pos == len(bs)
    return start, streams
