"""Pins of the latent-bitstream oracle (oracle/codec.py) against facts outside itself:
a hand-worked fixed-point example, the float64 ARM on a grid where fixed point is exact,
an independent Laplace CDF, range-coder round trips and code lengths, the wavefront
dependency rule by brute force."""
import math

import numpy as np
import pytest
import torch
from scipy import stats

from oracle import codec as C
from oracle import coolchic as oc

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ------------------------------------------------------------------ fixed-point ARM

def _arch(n, layers):
    return oc.Arch(arm_ctx=n, arm_layers=layers)


def test_fixed_arm_hand_example():
    """N = 2 (structure only), one LinR layer, worked by hand.

    W0 = [[0.5, 0], [0, -1]] (Q8 128, -256), b0 = [1/256, 0] (Q8 1, 0); context (3, 5)
    -> a = (768, 1280); z = ((384 + 128) >> 8 + 1... computed below step by step.
    """
    Q = {"arm.w0": np.array([[128, 0], [0, -256]]), "arm.b0": np.array([1, 0]),
         "arm.wout": np.array([[1, 0], [0, 3]]), "arm.bout": np.array([-100, 7])}
    arch = _arch(2, 1)
    # a = (3*256, 5*256) = (768, 1280)
    # z0 = ((128*768 + 128) >> 8) + 1 = (98432 >> 8) + 1 = 384 + 1 = 385
    # z1 = ((-256*1280 + 128) >> 8) + 0 = (-327552 >> 8) = -1280 (floor of -1279.5)
    # h = (768 + 385, 1280 + 0) = (1153, 1280)
    # mu = ((1*1153 + 128) >> 8) - 100 = (1281 >> 8) - 100 = 5 - 100 = -95
    # s  = ((3*1280 + 128) >> 8) + 7 = (3968 >> 8) + 7 = 15 + 7 = 22
    mu, s = C.arm_fixed(np.array([3, 5]), Q, arch)
    assert (int(mu), int(s)) == (-95, 22)


def test_fixed_arm_round_half_up():
    """(sum + 128) >> 8 rounds exact halves of a Q8 step up, for negative sums too.

    N = 1, W0 = 0 and b0 = h make the LinR layer output h for context 0; the output layer
    W = (1, -1) then sees the Q16 sums +h and -h."""
    arch = _arch(1, 1)
    for h, want in ((128, (1, 0)), (384, (2, -1)), (127, (0, 0)), (129, (1, -1))):
        Q = {"arm.w0": np.zeros((1, 1), np.int64), "arm.b0": np.array([h]),
             "arm.wout": np.array([[1], [-1]]), "arm.bout": np.zeros(2, np.int64)}
        got = tuple(int(v) for v in C.arm_fixed(np.array([0]), Q, arch))
        assert got == want, (h, got)


@pytest.mark.parametrize("n,layers", [(8, 2), (16, 1), (24, 2)])
def test_fixed_arm_equals_float_arm_on_dyadic_grid(n, layers):
    """Weights and biases on the 1/4 grid, integer contexts: every partial product of up
    to three layers lies on the 1/64 grid, so no fixed-point rounding happens and, with
    activations kept below the +-128 saturation, mu_q / 256, s_q / 256 equal the float64
    ARM (oracle.coolchic) exactly."""
    rng = np.random.default_rng(n * 10 + layers)
    arch = _arch(n, layers)
    named = {}
    for name, shape in oc.param_shapes(arch):
        if name.startswith("arm."):
            named[name] = rng.integers(-2, 3, size=shape) / 4.0
    ctx = rng.integers(-3, 4, size=(500, n))
    mu_q, s_q = C.arm_fixed(ctx, C.quantize_arm(named, arch), arch)
    P = {k: torch.tensor(v, dtype=oc.DT) for k, v in named.items()}
    mu, s = oc.arm_mlp(torch.tensor(ctx, dtype=oc.DT), P, arch)
    h = torch.tensor(ctx, dtype=oc.DT)
    for i in range(layers):      # no saturation anywhere
        h = h + torch.relu(h @ P[f"arm.w{i}"].T + P[f"arm.b{i}"])
        assert h.abs().max() < 128
    np.testing.assert_array_equal(mu_q / 256.0, mu.numpy())
    np.testing.assert_array_equal(s_q / 256.0, s.numpy())


def test_fixed_arm_context_clamp_and_int32_bound():
    """Contexts beyond +-128 act as +-128; the largest weights and activations the format
    allows keep every layer sum inside int32 (checked inside arm_fixed)."""
    arch = _arch(24, 2)
    rng = np.random.default_rng(9)
    Q = {}
    for name, shape in oc.param_shapes(arch):
        if name.startswith("arm."):
            lim = C.W_LIM if ".w" in name else C.ACT_LIM
            Q[name] = rng.choice([-lim, lim], size=shape).astype(np.int64)
    big = rng.choice([-10**6, 10**6, -129, 129, 500], size=(64, 24))
    clamped = np.clip(big, -C.CTX_LIM, C.CTX_LIM)
    a = C.arm_fixed(big, Q, arch)
    b = C.arm_fixed(clamped, Q, arch)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert np.abs(a[0]).max() <= C.ACT_LIM and np.abs(a[1]).max() <= C.ACT_LIM
    # the bound itself: N * W_LIM * ACT_LIM + rounding stays below 2^31
    assert 24 * C.W_LIM * C.ACT_LIM + 128 < 2 ** 31


def test_fixed_arm_close_to_float_arm():
    """General weights: the fixed-point ARM stays within a few Q8 steps of float64."""
    rng = np.random.default_rng(3)
    arch = _arch(24, 2)
    named = {name: rng.normal(0, 0.15, size=shape)
             for name, shape in oc.param_shapes(arch) if name.startswith("arm.")}
    ctx = rng.integers(-20, 21, size=(2000, 24))
    mu_q, s_q = C.arm_fixed(ctx, C.quantize_arm(named, arch), arch)
    P = {k: torch.tensor(v, dtype=oc.DT) for k, v in named.items()}
    mu, s = oc.arm_mlp(torch.tensor(ctx, dtype=oc.DT), P, arch)
    assert np.abs(mu_q / 256.0 - mu.numpy()).max() < 0.5
    assert np.abs(s_q / 256.0 - s.numpy()).max() < 0.5


def test_quantize_arm_clamps_and_rounds_half_even():
    arch = _arch(8, 1)
    named = {name: np.zeros(shape) for name, shape in oc.param_shapes(arch)
             if name.startswith("arm.")}
    named["arm.w0"][0, 0] = 1e9          # -> +2^11 (|w| <= 8)
    named["arm.w0"][0, 1] = 0.5 / 256     # half -> 0 (even)
    named["arm.w0"][0, 2] = 1.5 / 256     # -> 2
    named["arm.b0"][0] = -1e12           # -> -2^15
    Q = C.quantize_arm(named, arch)
    assert Q["arm.w0"][0, 0] == C.W_LIM
    assert Q["arm.w0"][0, 1] == 0 and Q["arm.w0"][0, 2] == 2
    assert Q["arm.b0"][0] == -C.ACT_LIM


# ------------------------------------------------------------------ tables

def test_table_index_boundaries():
    lo = C.LOGB_LO_Q
    t, m = C.table_index([0, 0, 0, 0, 0], [lo - 10**6, lo, lo + 31, lo + 32, 10**6])
    np.testing.assert_array_equal(t // C.NMU, [0, 0, 0, 1, C.NSCALE - 1])
    t, m = C.table_index([-1, 0, 31, 32, 255, 256, -256, -257], [lo] * 8)
    np.testing.assert_array_equal(m, [-1, 0, 0, 0, 0, 1, -1, -2])
    np.testing.assert_array_equal(t % C.NMU, [7, 0, 0, 1, 7, 0, 0, 7])
    assert C.LOGB_LO_Q == -1179
    # the last bin's upper edge passes the model's largest log-scale ln 1e3
    assert (C.LOGB_LO_Q + C.NSCALE * C.LOGB_STEP_Q) / 256.0 > math.log(1e3)


def test_tables_match_scipy_laplace():
    """Frequencies against scipy's Laplace CDF (an independent implementation)."""
    cum = C.build_tables()
    assert cum.shape == (C.NSCALE * C.NMU, C.NSYM + 1)
    assert (cum[:, 0] == 0).all() and (cum[:, -1] == C.TOTAL).all()
    freq = np.diff(cum, axis=1)
    assert freq.min() >= 1
    ks = np.arange(-C.A, C.A + 1)
    for t in range(0, C.NSCALE * C.NMU, 37):
        j, fi = divmod(t, C.NMU)
        b = math.exp(C.LOGB_LO_Q / 256 + (j + 0.5) / 8)
        f = (fi + 0.5) / 8
        law = stats.laplace(loc=f, scale=b)
        p = np.concatenate([[law.cdf(-C.A - 0.5)], law.cdf(ks + 0.5) - law.cdf(ks - 0.5),
                            [law.sf(C.A + 0.5)]])
        err = np.abs(freq[t] / C.TOTAL - p)
        assert err.max() <= 2.0 * C.NSYM / C.TOTAL, (t, err.max())
        # all but the symbol that took the remainder: within one count of the scaled mass
        rest_at = int(np.argmax(freq[t]))
        scaled = p * (C.TOTAL - C.NSYM)
        mask = np.ones(C.NSYM, bool)
        mask[rest_at] = False
        assert np.all(np.abs(freq[t][mask] - 1 - scaled[mask]) <= 1.0 + 1e-9)


def test_tables_mirror_symmetry():
    """Laplace(f) of symbol k equals Laplace(1 - f) of symbol 1 - k: fractional bins fi
    and NMU - 1 - fi mirror each other on the interior symbols."""
    cum = C.build_tables()
    freq = np.diff(cum, axis=1)
    for j in (0, 20, 40, 60, 92):
        for fi in range(C.NMU):
            a = freq[j * C.NMU + fi]
            b = freq[j * C.NMU + C.NMU - 1 - fi]
            # symbol k at index k + A + 1; interior k in [-A + 1, A - 1] maps to 1 - k
            for k in range(-C.A + 2, C.A - 1):
                if a[k + C.A + 1] != max(a) and b[1 - k + C.A + 1] != max(b):
                    assert abs(int(a[k + C.A + 1]) - int(b[1 - k + C.A + 1])) <= 1


# ------------------------------------------------------------------ range coder

def _random_freqs(rng, n):
    w = rng.exponential(1.0, n) ** 3 + 1e-6
    f = 1 + np.floor(w / w.sum() * (C.TOTAL - n)).astype(np.int64)
    f[np.argmax(f)] += C.TOTAL - f.sum()
    return f


@pytest.mark.parametrize("seed", range(4))
def test_range_coder_roundtrip_and_length(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 200))
    f = _random_freqs(rng, n)
    cum = np.concatenate([[0], np.cumsum(f)])
    syms = rng.choice(n, size=3000, p=f / f.sum())
    enc = C.RangeEncoder()
    for s in syms:
        enc.encode(int(cum[s]), int(f[s]))
    data = enc.finish()
    dec = C.RangeDecoder(data)
    got = []
    for _ in syms:
        t = dec.target()
        s = int(np.searchsorted(cum, t, side="right") - 1)
        dec.consume(int(cum[s]), int(f[s]))
        got.append(s)
    assert got == list(syms)
    ideal = float(-np.log2(f[syms] / C.TOTAL).sum())
    # the coder loses at most ~2^-7 bits per symbol to the truncated range (r = range >> 16
    # with range >= 2^24) plus the 32-bit flush
    assert 8 * len(data) <= ideal * (1 + 2.0 ** -7) + 40
    assert 8 * len(data) >= ideal - 8


def test_range_coder_carry_runs():
    """Byte-sized symbols: low often sits in [0xFF000000, 2^32), so 0xFF bytes are held
    back, and carries out of bit 32 ripple through them."""
    f = np.full(256, C.TOTAL // 256)
    cum = np.concatenate([[0], np.cumsum(f)])
    syms = np.random.default_rng(7).integers(0, 256, 20000)
    enc = C.RangeEncoder()
    carries, held = 0, 0
    orig = enc._shift_low

    def counting():
        nonlocal carries, held
        carries += enc.low >= 1 << 32
        held = max(held, enc.pending)
        orig()
    enc._shift_low = counting
    for s in syms:
        enc.encode(int(cum[s]), int(f[s]))
    data = enc.finish()
    assert carries > 0 and held >= 2      # carries, and a held-back 0xFF byte
    assert 20000 <= len(data) <= 20000 + 1   # 8 bits a symbol, first byte dropped, flush
    dec = C.RangeDecoder(data)
    for s in syms:
        t = dec.target()
        k = int(np.searchsorted(cum, t, side="right") - 1)
        dec.consume(int(cum[k]), int(f[k]))
        assert k == s


def test_symbol_escapes_roundtrip():
    cum = C.build_tables()
    rng = np.random.default_rng(11)
    ks = [0, 1, -1, C.A, -C.A, C.A + 1, -C.A - 1, C.A + 2, -C.A - 2, 1000, -1000,
          C.Y_LIM * 2, -C.Y_LIM * 2] + list(rng.integers(-300, 301, 400))
    tabs = rng.integers(0, C.NSCALE * C.NMU, len(ks))
    enc = C.RangeEncoder()
    for k, t in zip(ks, tabs):
        C.encode_symbol(enc, cum[t], int(k))
    dec = C.RangeDecoder(enc.finish())
    assert [C.decode_symbol(dec, cum[t]) for t in tabs] == [int(k) for k in ks]


# ------------------------------------------------------------------ wavefront

@pytest.mark.parametrize("n,lag", [(8, 3), (16, 4), (24, 4), (32, 5)])
def test_wavefront_lag_brute_force(n, lag):
    """Step(r, x) = x + lag r decodes every context position at an earlier step, and
    lag - 1 would not."""
    offs = oc.causal_offsets(n)
    assert C.wavefront_lag(offs) == lag
    for L, ok in ((lag, True), (lag - 1, False)):
        good = all(x + dx + L * (r + dy) < x + L * r
                   for r in range(6, 10) for x in range(6, 10) for dy, dx in offs)
        assert good == ok


# ------------------------------------------------------------------ bitstream

def _random_decoder(arch, rng):
    named = {}
    for name, shape in oc.param_shapes(arch):
        named[name] = rng.normal(0, 0.2, size=shape).astype(np.float32)
    named["arm.bout"] = np.array([0.1, 0.7], np.float32)
    return named


def _laplace_latents(H, W, arch, rng):
    out = []
    for l, (h, w) in enumerate(oc.level_shapes(H, W, arch.levels)):
        y = np.rint(rng.laplace(0, 0.3 + 0.5 * l, size=(h, w))).astype(np.int64)
        out.append(y)
    out[0][0, 0] = 5000          # escapes
    out[0][-1, -1] = -C.Y_LIM
    out[1][0, -1] = C.A + 1
    return out


@pytest.mark.parametrize("arch", [oc.Arch(arm_ctx=8, arm_layers=2, syn_hidden=8),
                                  oc.Arch(arm_ctx=24, arm_layers=2, up_kernel=4,
                                          up_per_level=False, syn_hidden=16, syn_res3x3=1)])
def test_bitstream_roundtrip(arch):
    rng = np.random.default_rng(arch.arm_ctx)
    H, W = 37, 53
    named = _random_decoder(arch, rng)
    y = _laplace_latents(H, W, arch, rng)
    bs = C.write_bitstream(H, W, arch, named, y)
    H2, W2, arch2, named2, y2 = C.read_bitstream(bs)
    assert (H2, W2, arch2) == (H, W, arch)
    for a, b in zip(y, y2):
        np.testing.assert_array_equal(a, b)
    Q = C.quantize_arm(named, arch)
    for name, _ in oc.param_shapes(arch):
        want = Q[name] / 256.0 if name.startswith("arm.") else named[name]
        np.testing.assert_array_equal(named2[name], want)
    start, streams = C.header_and_streams(bs)
    assert len(streams) == sum(h for h, _ in oc.level_shapes(H, W))


def test_rate_close_to_the_float_model():
    """Coded size of the latents against the float64 model's rate (eq. (1)'s R): the
    table quantisation (mu to 1/8, log-scale to 1/8) and the coder cost a few percent."""
    rng = np.random.default_rng(5)
    arch = oc.Arch(arm_ctx=8, arm_layers=2, syn_hidden=8)
    named = {name: rng.normal(0, 0.1, size=shape).astype(np.float32)
             for name, shape in oc.param_shapes(arch) if name.startswith("arm.")}
    named["arm.bout"] = np.array([0.3, 0.9], np.float32)     # mean 0.3, scale e^0.9
    h, w = 96, 96
    y = np.rint(rng.laplace(0.3, math.exp(0.9), size=(h, w))).astype(np.int64)
    Q = C.quantize_arm(named, arch)
    streams = C.encode_rows(y, Q, arch, C.build_tables())
    coded = 8 * sum(len(s) for s in streams)
    P = {k: torch.tensor(v, dtype=oc.DT) for k, v in named.items()}
    model = float(oc.total_bits([torch.tensor(y, dtype=oc.DT)], P, arch))
    # per-row overhead: at most one flush byte and a partial byte per substream
    assert abs(coded / model - 1) < 0.02
    assert coded <= model * 1.03 + 16 * h
