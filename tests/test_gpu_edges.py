"""Edge cases of the RIR kernels against the FP64 oracle (Sec. II.A
definition): the smallest lattice, RIRs of one or two samples, lengths at
the work-item window boundary, the shortest and longest filters (the 1-tap
Hann filter needs 11 Chebyshev terms, so it takes the generic term loop; the
255-tap one needs the widest sparse arrays), the 2-tap Lagrange
filter (linear interpolation), and mixed filters and orders in one call."""
import numpy as np
import pytest

import oracle
from paper_2104_13347_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1]


def rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def run(ism, rooms, variant, tol=1e-5, oracle_rooms=None):
    """The GPU path on `rooms` against the oracle on `oracle_rooms` (the
    same rooms unless given)."""
    import torch
    n_rirs, _ = ism.rir_batch_size(rooms)
    stats = torch.zeros(2 * n_rirs, dtype=torch.int64, device="cuda")
    h = ism.rir_batch(rooms, stats=stats, variant=variant)
    torch.cuda.synchronize()
    h = h.cpu().numpy().astype(np.float64)
    st = stats.view(-1, 2).cpu().numpy()
    ref, ost = oracle.rir_batch(rooms if oracle_rooms is None else oracle_rooms)
    o = j = 0
    for r, rr in zip(rooms, ref):
        L = r["rir_len"]
        for m in range(len(r["mics"])):
            g = h[o:o + L]
            if np.linalg.norm(rr[m]) == 0:
                assert not np.any(g)
            else:
                assert rel_l2(g, rr[m]) <= tol, (j, rel_l2(g, rr[m]))
            o += L
            j += 1
    np.testing.assert_array_equal(st[:, 0], ost[:, 1])
    np.testing.assert_array_equal(st[:, 1], ost[:, 2])


@pytest.mark.parametrize("variant", VARIANTS)
def test_order_zero_and_tiny_rirs(ism, variant):
    rooms = []
    for i, L in enumerate((1, 2, 3, 17)):
        rooms += wl.room_batch(1, seed=60 + i, order=0, rir_len=L, n_mics=2)
    # a source 0.3 m from the mic: the direct path lands in the first taps
    # (its delay is 14 samples: the 1- and 5-sample RIRs hold only the tails
    # of its filter, and take the direct per-tap kernel on the sparse path)
    rooms += [dict(dims=np.array([4.0, 3.0, 2.5]), beta=np.full(6, 0.9),
                   src=np.array([1.0, 1.0, 1.0]), mics=np.array([[1.3, 1.0, 1.0]]), fs=16000.0,
                   c=343.0, order=2, n_taps=81, fd_kind=0, rir_len=L) for L in (1, 5, 40)]
    run(ism, rooms, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_lengths_at_window_boundaries(ism, variant):
    rooms = []
    for i, L in enumerate((1023, 1024, 1025, 2047, 2048, 2049)):
        rooms += wl.room_batch(1, seed=70 + i, order=4, rir_len=L, n_mics=2)
    run(ism, rooms, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_extreme_filters(ism, variant):
    rooms = []
    for i, (kind, nt) in enumerate(((0, 1), (0, 3), (0, 255), (1, 2), (1, 4))):
        rooms += wl.room_batch(1, seed=80 + i, order=4, rir_len=3000, n_mics=2, n_taps=nt,
                               fd_kind=kind)
    run(ism, rooms, variant)


def test_sparse_term_counts():
    """Which filters above take the unrolled term loops: 8 terms for the
    Hann sinc from 33 taps up (255 included), 9 for 3 taps and 11 for the
    1-tap filter (its window is sharp, so the tap varies faster with the
    fraction) and exact counts for Lagrange filters -- so the generic loop
    is exercised too."""
    import paper_2104_13347_gb300 as ism
    assert ism.rir_filter_terms(0, 81) == 8 and ism.rir_filter_terms(0, 255) == 8
    assert ism.rir_filter_terms(0, 1) == 11 and ism.rir_filter_terms(0, 3) == 9
    assert ism.rir_filter_terms(1, 2) == 2 and ism.rir_filter_terms(1, 8) == 8


def test_tail_only_rirs_take_the_direct_kernel(ism):
    """RIRs that end before their direct arrival hold only filter tails; the
    sparse path routes them to the direct per-tap kernel, so with the same
    window they are bitwise those of the direct variant (and within the bar
    of the oracle); the other RIRs of the call stay on the sparse kernel."""
    import torch
    rooms = [dict(dims=np.array([6.0, 5.0, 3.0]), beta=np.full(6, 0.85),
                  src=np.array([1.0, 1.0, 1.5]), mics=np.array([[3.5, 2.0, 1.2], [1.2, 1.1, 1.5]]),
                  fs=16000.0, c=343.0, order=3, n_taps=81, fd_kind=0, rir_len=L)
             for L in (20, 100, 700)]
    hs = ism.rir_batch(rooms, window=256)
    hd = ism.rir_batch(rooms, window=256, variant=ism.RIR_DIRECT)
    torch.cuda.synchronize()
    hs, hd = hs.cpu().numpy(), hd.cpu().numpy()
    # mic 0 is 2.7 m away (126 samples): tail-only in the 20- and 100-sample
    # RIRs (the second holds the direct path's taps 86..99); mic 1 is 0.22 m
    # away (10 samples): its direct path is inside
    o = 0
    for L in (20, 100, 700):
        for m in range(2):
            seg = slice(o, o + L)
            if m == 0 and L < 126:
                np.testing.assert_array_equal(hs[seg], hd[seg])
                assert (L == 20) != bool(np.any(hs[seg]))
            o += L
    run(ism, rooms, 0)


@pytest.mark.parametrize("variant", VARIANTS)
def test_largest_lattice_order(ism, variant):
    """Order 200, the largest the ABI accepts (8 x 401^3 = 5.2e8 lattice
    images per RIR: per-axis tables of 802 entries, 643204 columns to sort
    per RIR), in rooms of about a metre with responses of 400 and 1600
    samples, Hann and Lagrange filters.  The oracle runs the delay-limited
    lattice instead, which holds every image able to reach the response
    (its own pin: a larger lattice changes nothing), so RIRs and the counts
    of contributing images and in-range taps must equal it."""
    rooms = []
    for i, (L, kind, taps) in enumerate([(400, 0, 81), (1600, 0, 81), (1600, 1, 8)]):
        rng = np.random.default_rng(300 + i)
        dims = np.array([1.0, 1.2, 0.9]) + rng.uniform(0, 0.2, 3)
        rooms.append(dict(dims=dims, beta=rng.uniform(0.5, 0.95, 6),
                          src=rng.uniform(0.2, 0.7, 3) * dims / dims.max(),
                          mics=np.stack([rng.uniform(0.25, 0.75, 3) * dims for _ in range(3)]),
                          fs=16000.0, c=343.0, order=200, n_taps=taps, fd_kind=kind,
                          rir_len=L))
    auto = [dict(r, order=-1) for r in rooms]  # ISM_ORDER_AUTO
    for r in auto:
        assert max(oracle.auto_order(r["dims"], r["src"], m, r["fs"], r["c"], r["n_taps"],
                                     r["rir_len"]) for m in r["mics"]) < 200
    run(ism, rooms, variant, oracle_rooms=auto)


@pytest.mark.parametrize("variant", VARIANTS)
def test_tail_only_rirs_of_wide_filters(ism, variant):
    """255-tap Hann filters on RIRs that end before the direct arrival, so
    that every sample is a far filter tail (both variants take the direct
    per-tap kernel for them): the outer taps' window values are ~1e-4 of the
    centre's, and must keep their relative precision (a window evaluated as
    1 + cos cancels there).  Rooms from a randomized sweep against the
    oracle: mics 1 mm from a wall, absorbing and rigid walls mixed."""
    rooms = [
        dict(dims=np.array([8.893839269383143, 10.506559043134592, 16.81623744945732]),
             beta=np.array([0.0, 1.0, 0.0, 0.888459665457403, 0.0, 0.3110977831570719]),
             src=np.array([6.450528485976667, 4.913054132597867, 10.390543488898375]),
             mics=np.array([[0.001, 3.2381923758825675, 11.647781849740037],
                            [4.580810968796418, 6.223670331673284, 16.815237449457317],
                            [3.020822382567682, 0.001, 11.259194720355325]]),
             fs=8000.0, c=343.0, order=-1, n_taps=255, fd_kind=0, rir_len=35),
        dict(dims=np.array([6.46555925860823, 19.18357269018504, 0.7633025218621846]),
             beta=np.array([0.4148920451030764, 0.7325607160274136, 0.0, 0.4594006983848494,
                            0.5676990312042093, 0.0]),
             src=np.array([3.802768292943413, 15.90782723262708, 0.5777257551062134]),
             mics=np.array([[1.6813341875345282, 5.075864370062916, 0.5445760219183458],
                            [3.625247770177144, 19.18257269018504, 0.05969707331769491]]),
             fs=16000.0, c=343.0, order=-1, n_taps=255, fd_kind=0, rir_len=389),
    ]
    run(ism, rooms, variant)
