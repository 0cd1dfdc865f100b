"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

arXiv 2104.13347 prints no RIR values, so each oracle function is pinned by
mathematics the paper's method fixes (Sec. II.A): the image set produced by
explicit successive mirror reflections, closed forms (an exact integer delay,
a single direct path), invariants (reciprocity, mirror symmetry), properties
of the fractional-delay filters (band-limited interpolation, Lagrange
polynomial exactness), an FFT convolution, and statistics of the noise
generator (Sec. III.A).  A plausible slip in the oracle (a dropped term, a
wrong sign or index, a swapped wall) fails at least one of these.
"""
import math

import numpy as np
import pytest

import oracle

FS, C = 16000.0, 343.0


# ---------------------------------------------------------------------------
# Image set: brute-force mirror reflections vs the lattice (Sec. II.A)
# ---------------------------------------------------------------------------

def mirror_images(dims, src, depth):
    """Every image reachable by reflecting the source across the six wall
    planes, breadth first, keeping the first (shortest) path to each
    position.  Returns {position (rounded key): (position, hits[6])} where
    hits counts reflections per wall (x0, x1, y0, y1, z0, z1)."""
    L = np.asarray(dims, float)
    start = (tuple(np.asarray(src, float)), (0,) * 6)
    seen = {tuple(np.round(start[0], 9)): start}
    frontier = [start]
    for _ in range(depth):
        nxt = []
        for pos, hits in frontier:
            for wall in range(6):
                ax, side = divmod(wall, 2)
                p = list(pos)
                p[ax] = -p[ax] if side == 0 else 2.0 * L[ax] - p[ax]
                key = tuple(np.round(p, 9))
                if key in seen:
                    continue
                h = list(hits)
                h[wall] += 1
                item = (tuple(p), tuple(h))
                seen[key] = item
                nxt.append(item)
        frontier = nxt
    return seen


@pytest.mark.parametrize("order", [0, 1, 2])
def test_lattice_equals_mirror_images(order):
    dims = [3.1, 2.3, 1.7]
    src = [0.7, 1.9, 0.4]
    mic = [2.2, 0.6, 1.3]
    beta = [0.9, 0.8, 0.7, 0.6, 0.5, 0.4]
    im = oracle.images(dims, beta, src, mic, FS, C, order)
    assert im["count"] == 8 * (2 * order + 1) ** 3

    # The lattice of order N is the set of images inside the box
    # (-(2N+1)L, (2N+1)L) on each axis.
    bf = mirror_images(dims, src, depth=3 * (2 * order + 1) + 1)
    box = (2 * order + 1) * np.asarray(dims)
    ref = []
    for pos, hits in bf.values():
        p = np.asarray(pos)
        if np.all(np.abs(p) < box):
            d = np.linalg.norm(p - np.asarray(mic))
            gain = np.prod([b ** k for b, k in zip(beta, hits)])
            ref.append((d, gain))
    key = lambda t: (round(t[0], 9), t[1])
    ref.sort(key=key)
    got = sorted(zip(im["d"], im["amp"] * 4.0 * np.pi * im["d"]), key=key)
    assert len(ref) == len(got) == im["count"]
    ref, got = np.asarray(ref), np.asarray(got)
    np.testing.assert_allclose(got[:, 0], ref[:, 0], rtol=1e-13)
    np.testing.assert_allclose(got[:, 1], ref[:, 1], rtol=1e-12)


def test_delay_split_definition():
    """tau = d fs / c, k0 the nearest integer, f = tau - k0 in [-1/2, 1/2]."""
    dims, src, mic = [6.0, 5.0, 3.0], [1.1, 2.2, 1.3], [4.4, 3.1, 1.9]
    im = oracle.images(dims, [0.7] * 6, src, mic, 48000.0, C, 4)
    d_np = np.empty(im["count"])
    for i, (u, v, w, l, m, n) in enumerate(im["idx"]):
        p = np.array([(1 - 2 * u) * src[0] + 2 * l * dims[0],
                      (1 - 2 * v) * src[1] + 2 * m * dims[1],
                      (1 - 2 * w) * src[2] + 2 * n * dims[2]])
        d_np[i] = np.linalg.norm(p - np.asarray(mic))
    np.testing.assert_allclose(im["d"], d_np, rtol=1e-14)
    np.testing.assert_allclose(im["tau"], d_np * 48000.0 / C, rtol=1e-14)
    assert np.all(np.abs(im["f"]) <= 0.5)
    np.testing.assert_array_equal(im["k0"] + im["f"], im["tau"])


def test_image_density_matches_room_volume():
    """Images are one per room volume: count(d < R) ~ (4/3) pi R^3 / V."""
    dims = [5.0, 4.0, 3.0]
    im = oracle.images(dims, [0.8] * 6, [1.3, 2.1, 0.9], [3.6, 1.2, 2.2], FS, C, 10)
    R = 50.0
    expect = 4.0 / 3.0 * math.pi * R ** 3 / np.prod(dims)
    got = np.count_nonzero(im["d"] < R)
    assert abs(got - expect) / expect < 0.02


# ---------------------------------------------------------------------------
# Fractional-delay filters
# ---------------------------------------------------------------------------

def test_hann_sinc_zero_delay_is_kronecker():
    taps = oracle.hann_sinc_taps(0.0, 81)
    ref = np.zeros(81)
    ref[40] = 1.0
    np.testing.assert_array_equal(taps, ref)


@pytest.mark.parametrize("f", [-0.5, -0.31, -0.02, 0.17, 0.4999])
def test_hann_sinc_is_a_delay(f):
    """Applied to samples of a band-limited cosine, the taps reproduce the
    cosine at the fractional offset -f (a delay by f, not an advance)."""
    taps = oracle.hann_sinc_taps(f, 81)
    j = np.arange(-40, 41)
    rng = np.random.default_rng(7)
    for omega in (0.05 * np.pi, 0.2 * np.pi, 0.4 * np.pi):
        phi = rng.uniform(0, 2 * np.pi)
        got = np.dot(taps, np.cos(-omega * j + phi))
        assert abs(got - np.cos(-omega * f + phi)) < 2e-3
    # DC gain
    assert abs(taps.sum() - 1.0) < 2e-3


def test_hann_sinc_mirror_symmetry():
    a = oracle.hann_sinc_taps(0.23, 81)
    b = oracle.hann_sinc_taps(-0.23, 81)
    np.testing.assert_allclose(a, b[::-1], rtol=0, atol=1e-16)


def test_hann_sinc_three_taps_closed_form():
    """The window's width and centring (reading D2: w(t) = (1 + cos(pi t /
    (H + 1))) / 2 on t = j - f) in closed form.  Three taps (H = 1) at the
    half-sample delay f = 1/2 sit at t = -3/2, -1/2, 1/2, where sin(pi t) =
    1, -1, 1, cos(pi t / 2) = -sqrt(2)/2, sqrt(2)/2, sqrt(2)/2, so the taps
    are -(1 - sqrt(2)/2) / (3 pi), (1 + sqrt(2)/2) / pi, (1 + sqrt(2)/2) / pi.
    A window of width H instead of H + 1 would give 1/pi and -1/(3 pi)."""
    r2 = math.sqrt(2.0) / 2.0
    ref = np.array([-(1.0 - r2) / (3.0 * math.pi), (1.0 + r2) / math.pi,
                    (1.0 + r2) / math.pi])
    np.testing.assert_allclose(ref, [-0.0310769357, 0.5433889652, 0.5433889652], atol=1e-10)
    np.testing.assert_allclose(oracle.hann_sinc_taps(0.5, 3), ref, rtol=0, atol=1e-15)


def test_hann_sinc_81_taps_by_hand():
    """Two taps of the 81-tap filter (H = 40) at f = 1/2, written out from
    the reading's formula: the centre tap j = 0 (t = -1/2, sinc = 2/pi) is
    (1 + cos(pi / 82)) / pi, the last tap j = 40 (t = 79/2, sin(pi t) = -1)
    is -(1 + cos(79 pi / 82)) / (79 pi)."""
    taps = oracle.hann_sinc_taps(0.5, 81)
    centre = (1.0 + math.cos(math.pi / 82.0)) / math.pi
    last = -(1.0 + math.cos(79.0 * math.pi / 82.0)) / (79.0 * math.pi)
    assert abs(taps[40] - centre) <= 1e-13 * abs(centre)
    assert abs(taps[80] - last) <= 1e-12 * abs(last)


def test_hann_sinc_short_filter_window_positive():
    """Window 0.5(1+cos(pi t/(H+1))) stays positive on every tap, so every
    tap has the sign of the sinc."""
    f = 0.37
    for n in (3, 9, 81):
        H = (n - 1) // 2
        taps = oracle.hann_sinc_taps(f, n)
        t = np.arange(-H, H + 1) - f
        assert np.all(np.sign(taps) == np.sign(np.sinc(t)))


@pytest.mark.parametrize("D", [3.0, 3.25, 3.5, 3.999])
def test_lagrange_exact_for_polynomials(D):
    taps = oracle.lagrange_taps(D, 8)
    j = np.arange(8, dtype=float)
    for p in range(8):
        assert abs(np.dot(taps, j ** p) - D ** p) <= 1e-10 * max(1.0, D ** p)
    if D == 3.0:
        ref = np.zeros(8)
        ref[3] = 1.0
        np.testing.assert_array_equal(taps, ref)


# ---------------------------------------------------------------------------
# Whole RIRs
# ---------------------------------------------------------------------------

def test_exact_integer_delay_is_delta():
    """fs/c = 64 exactly, mic 1 m from the source along x, order 0 and
    anechoic walls: h = delta[n - 64] / (4 pi), bit for bit."""
    h = oracle.rir([5, 4, 3], [0.0] * 6, [2.0, 1.5, 1.5], [3.0, 1.5, 1.5], 16384.0, 256.0,
                   0, 81, oracle.FD_HANN_SINC, 256)
    ref = np.zeros(256)
    ref[64] = 1.0 / (4.0 * np.pi)
    np.testing.assert_array_equal(h, ref)


def test_single_direct_path_closed_form():
    src, mic = np.array([1.27, 2.31, 1.05]), np.array([3.93, 1.12, 2.01])
    d = np.linalg.norm(src - mic)
    tau = d * FS / C
    k0 = int(np.rint(tau))
    f = tau - k0
    h = oracle.rir([5, 4, 3], [0.0] * 6, src, mic, FS, C, 0, 81, oracle.FD_HANN_SINC, 1024)
    ref = np.zeros(1024)
    ref[k0 - 40:k0 + 41] = oracle.hann_sinc_taps(f, 81) / (4 * np.pi * d)
    np.testing.assert_allclose(h, ref, rtol=1e-12, atol=1e-18)
    # band-limited peak sits at the delay: the continuous interpolant's
    # maximum is within a fraction of a sample of tau
    fine = np.linspace(-1, 1, 2001)
    n = np.arange(k0 - 40, k0 + 41)
    recon = [np.dot(h[n], np.sinc(k0 + x - n)) for x in fine]
    assert abs(k0 + fine[int(np.argmax(recon))] - tau) < 2e-2


def test_reciprocity():
    dims, beta = [4.3, 3.7, 2.9], [0.9, 0.6, 0.8, 0.7, 0.5, 0.95]
    a, b = [1.1, 2.2, 0.7], [3.0, 1.4, 2.1]
    h1 = oracle.rir(dims, beta, a, b, FS, C, 4, 81, oracle.FD_HANN_SINC, 2048)
    h2 = oracle.rir(dims, beta, b, a, FS, C, 4, 81, oracle.FD_HANN_SINC, 2048)
    assert np.linalg.norm(h1 - h2) / np.linalg.norm(h1) < 1e-12


def test_mirror_symmetry_of_room():
    """Mirroring x -> Lx - x and swapping the two x walls maps image (u=1, l)
    to (u=1, 1-l), so the order-N lattice is only mirror-symmetric inside its
    outer shell: the RIR is cut (800 samples = 17 m) before the shell."""
    dims, beta = [4.3, 3.7, 2.9], [0.9, 0.6, 0.8, 0.7, 0.5, 0.95]
    a, b = np.array([1.1, 2.2, 0.7]), np.array([3.0, 1.4, 2.1])
    h1 = oracle.rir(dims, beta, a, b, FS, C, 4, 81, oracle.FD_HANN_SINC, 800)
    am, bm = a.copy(), b.copy()
    am[0], bm[0] = dims[0] - a[0], dims[0] - b[0]
    beta_m = [beta[1], beta[0]] + beta[2:]
    h2 = oracle.rir(dims, beta_m, am, bm, FS, C, 4, 81, oracle.FD_HANN_SINC, 800)
    assert np.linalg.norm(h1 - h2) / np.linalg.norm(h1) < 1e-12


def test_rir_is_sum_over_mirror_images():
    """Order 1 RIR equals the direct sum over brute-force mirror images."""
    dims, beta = [3.1, 2.3, 1.7], [0.9, 0.8, 0.7, 0.6, 0.5, 0.4]
    src, mic = [0.7, 1.9, 0.4], [2.2, 0.6, 1.3]
    bf = mirror_images(dims, src, depth=10)
    box = 3 * np.asarray(dims)
    Lh = 512
    ref = np.zeros(Lh)
    for pos, hits in bf.values():
        p = np.asarray(pos)
        if not np.all(np.abs(p) < box):
            continue
        d = np.linalg.norm(p - np.asarray(mic))
        g = np.prod([b ** k for b, k in zip(beta, hits)]) / (4 * np.pi * d)
        tau = d * FS / C
        k0 = int(np.rint(tau))
        taps = oracle.hann_sinc_taps(tau - k0, 81)
        for j in range(-40, 41):
            if 0 <= k0 + j < Lh:
                ref[k0 + j] += g * taps[j + 40]
    h = oracle.rir(dims, beta, src, mic, FS, C, 1, 81, oracle.FD_HANN_SINC, Lh)
    np.testing.assert_allclose(h, ref, rtol=1e-11, atol=1e-15)


def test_stats_count_taps_in_range():
    dims = [5, 4, 3]
    src, mic = [1.2, 1.5, 1.1], [3.3, 2.2, 1.7]
    Lh = 700
    h, st = oracle.rir(dims, [0.8] * 6, src, mic, FS, C, 3, 81, oracle.FD_HANN_SINC, Lh,
                       return_stats=True)
    im = oracle.images(dims, [0.8] * 6, src, mic, FS, C, 3)
    lo = np.clip(im["k0"] - 40, 0, Lh)
    hi = np.clip(im["k0"] + 41, 0, Lh)
    taps = np.maximum(hi - lo, 0)
    assert st["images"] == im["count"] == 8 * 7 ** 3
    assert st["taps"] == int(taps.sum())
    assert st["contributing"] == int(np.count_nonzero(taps))


def test_lagrange_rir_direct_path():
    src, mic = np.array([1.27, 2.31, 1.05]), np.array([3.93, 1.12, 2.01])
    d = np.linalg.norm(src - mic)
    tau = d * FS / C
    fl = int(np.floor(tau))
    h = oracle.rir([5, 4, 3], [0.0] * 6, src, mic, FS, C, 0, 8, oracle.FD_LAGRANGE, 512)
    nz = np.nonzero(h)[0]
    assert nz.min() == fl - 3 and nz.max() == fl + 4
    # the 8 taps interpolate any cubic exactly at the delay: sum_j h_j p(j) = a p(tau)
    a = 1 / (4 * np.pi * d)
    n = np.arange(fl - 3, fl + 5, dtype=float)
    p = lambda x: 0.3 - 0.02 * x + 1e-4 * x ** 2 - 1e-6 * x ** 3
    assert abs(np.dot(h[fl - 3:fl + 5], p(n)) - a * p(tau)) < 1e-12


# ---------------------------------------------------------------------------
# Convolution
# ---------------------------------------------------------------------------

def test_convolution_matches_fft():
    from scipy.signal import fftconvolve
    rng = np.random.default_rng(3)
    h = rng.standard_normal(777)
    s = rng.standard_normal(1500)
    y = oracle.convolve(h, s)
    ref = fftconvolve(h, s)
    assert y.shape == (1500 + 777 - 1,)
    assert np.max(np.abs(y - ref)) < 1e-11 * np.max(np.abs(ref))
    ts = np.array([0, 5, 776, 777, 1499, 1500, 2275])
    np.testing.assert_allclose(oracle.convolve_at(h, s, ts), y[ts], rtol=0, atol=0)


def test_convolution_delta_and_linearity():
    rng = np.random.default_rng(4)
    s = rng.standard_normal(300)
    h = np.zeros(50)
    h[17] = 1.0
    y = oracle.convolve(h, s)
    np.testing.assert_array_equal(y[17:317], s)
    assert not np.any(y[:17]) and not np.any(y[317:])
    h2 = rng.standard_normal(50)
    s2 = rng.standard_normal(300)
    lin = oracle.convolve(h2, 2.0 * s + 3.0 * s2)
    np.testing.assert_allclose(lin, 2.0 * oracle.convolve(h2, s) + 3.0 * oracle.convolve(h2, s2),
                               rtol=1e-12, atol=1e-12)


def test_convolve_batch_matches_single():
    rng = np.random.default_rng(5)
    hs = [rng.standard_normal((3, 64)), rng.standard_normal((2, 40))]
    ss = [rng.standard_normal(100), rng.standard_normal(77)]
    ys = oracle.convolve_batch(hs, ss, n_threads=2)
    for H, s, Y in zip(hs, ss, ys):
        for m in range(H.shape[0]):
            np.testing.assert_array_equal(Y[m], oracle.convolve(H[m], s))


# ---------------------------------------------------------------------------
# Noise (Sec. III.A)
# ---------------------------------------------------------------------------

def test_splitmix64_published_sequence():
    """First outputs of SplitMix64 seeded with 0, as published with the
    generator's reference implementation."""
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 2) == 0x06C45D188009454F


def test_noise_uniforms_and_gaussian():
    """Uniforms of the noise streams are uniform, the even and odd samples
    of a pair are the two Box--Muller branches of the pair's uniforms
    (independent standard normals), and different streams are uncorrelated."""
    from scipy import stats
    u1, u2 = oracle.uniforms(1234, 7, 3, 0, 200000)
    assert u1.min() > 0 and u1.max() < 1 and u2.min() >= 0 and u2.max() < 1
    for u in (u1, u2):
        hist, _ = np.histogram(u, bins=64, range=(0, 1))
        assert stats.chisquare(hist).pvalue > 1e-4
    r = np.sqrt(-2 * np.log(u1))
    zc, zs = r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)
    for z in (zc, zs):
        assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(zc, zs)[0, 1]) < 0.01
    assert abs(np.corrcoef(u1, u2)[0, 1]) < 0.01
    for k in (0, 11, 12345):
        assert abs(oracle.gauss(1234, 7, 3, 2 * k) - zc[k]) < 1e-15
        assert abs(oracle.gauss(1234, 7, 3, 2 * k + 1) - zs[k]) < 1e-15
    # the pair's uniforms are the top two 24-bit fields of one counter output
    b = oracle.splitmix64(oracle.splitmix64(1234, 7 * 65536 + 3), 11)
    assert u1[11] == ((b >> 40) + 0.5) / 2 ** 24 and u2[11] == ((b >> 16) & 0xFFFFFF) / 2 ** 24
    v1, _ = oracle.uniforms(1234, 7, 4, 0, 200000)
    assert abs(np.corrcoef(u1, v1)[0, 1]) < 0.01


def test_noise_reaches_snr():
    rng = np.random.default_rng(9)
    y = rng.standard_normal((8, 20000)) * 0.3
    clean = y.copy()
    noisy, sigma = oracle.add_noise(y, 12.5, 99, 5)
    n = noisy - clean
    p_sig = np.mean(clean ** 2)
    assert abs(sigma - math.sqrt(p_sig / 10 ** 1.25)) < 1e-15
    snr = 10 * np.log10(p_sig / np.mean(n ** 2))
    assert abs(snr - 12.5) < 0.05


# ---------------------------------------------------------------------------
# Delay-limited image sets (Sec. II.A: every reflection arriving within the
# reverberation time is kept; the paper's 7 x 10 x 3.7 m room at RT 0.5 s
# needs reflections up to about the 60th order, more than 80000 images).
# ---------------------------------------------------------------------------

def test_auto_order_covers_every_image_within_reach():
    """No image that can put a tap into [0, Lh) lies outside the automatic
    lattice (checked on a lattice two orders larger), and the RIR does not
    change when the lattice grows."""
    dims, src, mic = np.array([4.3, 3.1, 2.7]), np.array([1.1, 2.2, 0.9]), np.array([3.0, 0.7, 1.8])
    beta = np.array([0.9, 0.7, 0.8, 0.95, 0.6, 0.85])
    fs, c, L, taps = 16000.0, 343.0, 1500, 81
    N = oracle.auto_order(dims, src, mic, fs, c, taps, L)
    reach = (L + taps) * c / fs
    big = oracle.images(dims, beta, src, mic, fs, c, N + 2)
    far = np.abs(big["idx"][:, 3:]).max(axis=1) > N
    assert not np.any(far & (big["d"] <= reach))
    h_auto, st_auto = oracle.rir(dims, beta, src, mic, fs, c, -1, taps, 0, L, return_stats=True)
    h_big, st_big = oracle.rir(dims, beta, src, mic, fs, c, N + 3, taps, 0, L, return_stats=True)
    np.testing.assert_array_equal(h_auto, h_big)
    assert st_auto["contributing"] == st_big["contributing"] and st_auto["taps"] == st_big["taps"]
    assert st_auto["images"] == 8 * (2 * N + 1) ** 3


def test_paper_room_images_within_rt():
    """The paper's classroom (7 x 10 x 3.7 m, array at [4, 6, 1.5], RT 0.5 s,
    44.1 kHz): more than 80000 images arrive within the RT, with reflection
    orders up to the mid-fifties (the paper quotes 'up to the 60th order')."""
    dims, mic, src = np.array([7.0, 10.0, 3.7]), np.array([4.0, 6.0, 1.5]), np.array([6.0, 6.5, 1.6])
    fs, c, rt = 44100.0, 343.0, 0.5
    N = oracle.auto_order(dims, src, mic, fs, c, 81, int(rt * fs))
    im = oracle.images(dims, np.full(6, 0.9), src, mic, fs, c, N)
    keep = im["d"] <= c * rt
    u, v, w, l, m, n = (im["idx"][:, i] for i in range(6))
    refl = np.abs(l - u) + np.abs(l) + np.abs(m - v) + np.abs(m) + np.abs(n - w) + np.abs(n)
    assert 80000 < keep.sum() < 90000
    assert 50 <= refl[keep].max() <= 60
    # density check: the count matches the sphere volume over the room volume
    assert abs(keep.sum() / (4 / 3 * np.pi * (c * rt) ** 3 / np.prod(dims)) - 1) < 0.01


# ---------------------------------------------------------------------------
# Energy decay of the image sum (Sec. II.A: each image carries the cumulated
# damping of the walls it met) and the walls drawn from an RT60
# ---------------------------------------------------------------------------

DECAY_ROOMS = [((5.0, 4.0, 3.0), (1.2, 1.1, 1.3), (3.6, 2.7, 1.6), 0.25),
               ((7.0, 10.0, 3.7), (2.0, 3.0, 1.2), (4.0, 6.0, 1.5), 0.5)]


def schroeder_t20(h, fs):
    """T20 of a RIR: the Schroeder backward-integrated energy fitted by a
    line between -5 and -25 dB, extrapolated to 60 dB."""
    e = np.cumsum((np.asarray(h, np.float64) ** 2)[::-1])[::-1]
    lev = 10.0 * np.log10(e / e[0])
    i5, i25 = int(np.argmax(lev <= -5.0)), int(np.argmax(lev <= -25.0))
    t = np.arange(len(h)) / fs
    return -60.0 / np.polyfit(t[i5:i25], lev[i5:i25], 1)[0]


def test_lattice_damping_gives_eyring_initial_decay():
    """A ray leaving the receiver along u meets the x walls |u_x| / Lx times
    per metre (y, z likewise); over the sphere that averages to S / (4V), the
    inverse mean free path.  The oracle's images in a shell well inside the
    lattice carry beta^n / (4 pi d) with an integer n whose mean per metre is
    that value, so with Eyring walls for RT60 the energy of the image sum
    starts to fall at 60 dB per RT60."""
    from paper_2104_13347_gb300 import workloads as wl
    for dims, src, mic, rt in DECAY_ROOMS:
        L = np.array(dims)
        V, S = np.prod(L), 2 * (L[0] * L[1] + L[0] * L[2] + L[1] * L[2])
        beta = wl.eyring_beta(dims, rt)
        N = 14
        im = oracle.images(dims, np.full(6, beta), src, mic, 8000.0, C, N)
        d = im["d"]
        shell = (d > 40.0) & (d < (2 * N - 1) * L.min())
        assert shell.sum() > 10000
        n = np.log(im["amp"][shell] * 4 * np.pi * d[shell]) / math.log(beta)
        np.testing.assert_allclose(n, np.round(n), atol=1e-8)
        rate = np.mean(n / d[shell])
        assert abs(rate / (S / (4 * V)) - 1) < 3e-3
        slope_db_per_s = 10 * math.log10(beta ** 2) * C * rate
        assert abs(slope_db_per_s * rt / -60.0 - 1) < 3e-3


def test_decay_time_scales_with_log_beta():
    """For a fixed room and positions the image sum's energy depends on time
    only through (-ln beta) t, so the decay times of RIRs with Sabine and
    with Eyring walls for the same RT60 stand in the ratio ln beta_S /
    ln beta_E (the Eyring walls reflect more)."""
    from paper_2104_13347_gb300 import workloads as wl
    fs = 8000.0
    for dims, src, mic, rt in DECAY_ROOMS:
        n = int(math.ceil(1.5 * rt * fs))
        bs, be = wl.sabine_beta(dims, rt), wl.eyring_beta(dims, rt)
        hs = oracle.rir(dims, np.full(6, bs), src, mic, fs, C, -1, rir_len=n)
        he = oracle.rir(dims, np.full(6, be), src, mic, fs, C, -1, rir_len=n)
        ratio = schroeder_t20(he, fs) / schroeder_t20(hs, fs)
        assert abs(ratio / (math.log(bs) / math.log(be)) - 1) < 0.03


# ---------------------------------------------------------------------------
# Training frames (Sec. II.B: 1024-sample multichannel windows; Sec. III.A:
# measurement noise at a drawn SNR)
# ---------------------------------------------------------------------------

def test_frame_is_the_slice_with_zero_padding():
    y = np.random.default_rng(3).standard_normal((4, 300))
    for t0 in (0, 17, -50, 280, 400, -2000):
        f, sig = oracle.frame(y, t0, 96, math.inf, 1, 2)
        assert sig == 0.0
        exp = np.zeros((4, 96))
        for i in range(96):
            if 0 <= t0 + i < 300:
                exp[:, i] = y[:, t0 + i]
        np.testing.assert_array_equal(f, exp)
    f2, _ = oracle.frame(y, 5, 96, math.nan, 1, 2)
    np.testing.assert_array_equal(f2, y[:, 5:101])


def test_frame_noise_snr_and_streams():
    """The added noise is sigma times the library's Gaussian stream of the
    frame (one stream per mic, sample index from the frame start) and
    reaches the requested SNR against the frame's own power."""
    rng = np.random.default_rng(4)
    y = rng.standard_normal((7, 5000)) * np.linspace(0.2, 1.0, 5000)
    clean, _ = oracle.frame(y, 1200, 1024, math.inf, 9, 33)
    noisy, sig = oracle.frame(y, 1200, 1024, 13.0, 9, 33)
    p = np.mean(clean ** 2)
    assert abs(sig - math.sqrt(p / 10 ** 1.3)) <= 1e-15 * sig
    z = (noisy - clean) / sig
    for m, i in ((0, 0), (3, 511), (6, 1023)):
        assert abs(z[m, i] - oracle.gauss(9, 33, m, i)) < 1e-9
    # SNR of the realised noise (7168 samples: within ~0.2 dB)
    assert abs(10 * np.log10(p / np.mean((noisy - clean) ** 2)) - 13.0) < 0.25
    # silence stays silent whatever the SNR
    z0, s0 = oracle.frame(np.zeros((2, 50)), 0, 32, 10.0, 1, 1)
    assert s0 == 0.0 and not np.any(z0)
