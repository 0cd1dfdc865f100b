"""The seeded input generators (CPU): the paper's dataset geometry
(Sec. II.A and III.A: UMA-8 array of 7 mics, sources in a torus of central
radius 2 m, dR 0.5 m, dphi 7 degrees, the 7 x 10 x 3.7 m and 5 x 5 x 4 m
rooms at RT 0.5 s, fs 44.1 kHz) and the reproducibility of every draw."""
import numpy as np
import pytest

from paper_2104_13347_gb300 import workloads as wl


def test_uma8_geometry():
    m = wl.uma8_array(np.array([4.0, 6.0, 1.5]))
    assert m.shape == (7, 3)
    np.testing.assert_allclose(m[0], [4.0, 6.0, 1.5])
    r = np.linalg.norm(m[1:] - m[0], axis=1)
    np.testing.assert_allclose(r, 0.04, rtol=1e-12)
    np.testing.assert_allclose(m[:, 2], 1.5)
    # six mics 60 degrees apart
    ang = np.sort(np.mod(np.arctan2(m[1:, 1] - 6.0, m[1:, 0] - 4.0), 2 * np.pi))
    np.testing.assert_allclose(np.diff(ang), np.pi / 3, atol=1e-12)


@pytest.mark.parametrize("room", [1, 2])
def test_torus_sources_in_the_room(room):
    dims, ctr = wl.PAPER_ROOMS[room]
    s = wl.torus_sources(4000, ctr, dims, seed=3)
    d = s - ctr
    r = np.linalg.norm(d, axis=1)
    assert r.min() >= 1.5 - 1e-12 and r.max() <= 2.5 + 1e-12
    el = np.degrees(np.arcsin(d[:, 2] / r))
    assert np.abs(el).max() <= 7.0 + 1e-9
    assert np.all(s > 0.1) and np.all(s < dims - 0.1)
    # azimuths cover the circle (room 1 fits the whole torus)
    if room == 1:
        az = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2 * np.pi)
        hist, _ = np.histogram(az, bins=12, range=(0, 2 * np.pi))
        assert hist.min() > 0.6 * hist.mean()


def test_paper_dataset_requests():
    a = wl.paper_dataset(16, room=1, seed=11)
    b = wl.paper_dataset(16, room=1, seed=11)
    assert len(a) == 16
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x["src"], y["src"])
    r = a[0]
    assert r["fs"] == 44100.0 and r["rir_len"] == 22050 and r["order"] == -1
    assert r["mics"].shape == (7, 3)
    # Sabine walls for RT 0.5 s in the 7 x 10 x 3.7 m room
    L = wl.PAPER_ROOMS[1][0]
    V, S = np.prod(L), 2 * (L[0] * L[1] + L[0] * L[2] + L[1] * L[2])
    assert abs(r["beta"][0] ** 2 - (1 - 0.161 * V / (S * 0.5))) < 1e-12
    lag = wl.paper_dataset(2, room=2, fd_kind=wl.FD_LAGRANGE, n_taps=8)
    assert lag[0]["fd_kind"] == 1 and lag[0]["n_taps"] == 8


def test_eyring_walls():
    """Eyring's alpha = 1 - exp(-0.161 V / (S RT60)) lies below Sabine's
    0.161 V / (S RT60) (more reflective walls for the same RT60), tends to it
    as the absorption vanishes, and stays inside (0, 1) where Sabine's
    clamps; the generators take either law and keep Sabine by default."""
    dims = np.array([5.0, 4.0, 3.0])
    for rt in (0.1, 0.3, 1.0, 3.0):
        be, bs = wl.eyring_beta(dims, rt), wl.sabine_beta(dims, rt)
        assert 0.0 <= bs < be < 1.0
    a = lambda b: 1.0 - b * b
    assert abs(a(wl.eyring_beta(dims, 100.0)) / a(wl.sabine_beta(dims, 100.0)) - 1) < 2e-3
    # RT60 so short that Sabine's alpha passes 1: Sabine gives beta 0, Eyring a wall
    assert wl.sabine_beta(dims, 0.05) == 0.0 and 0.0 < wl.eyring_beta(dims, 0.05) < 1.0
    assert wl.wall_beta(dims, 0.4, "eyring") == wl.eyring_beta(dims, 0.4)
    with pytest.raises(ValueError):
        wl.wall_beta(dims, 0.4, "lehmann")
    r_s, r_e = wl.ragged_batch(8, seed=3), wl.ragged_batch(8, seed=3, walls="eyring")
    for x, y in zip(r_s, r_e):
        assert x["beta"][0] == wl.sabine_beta(x["dims"], x["rt60"])
        assert y["beta"][0] == wl.eyring_beta(y["dims"], y["rt60"])
        assert x["rir_len"] == y["rir_len"] and x["order"] == y["order"]
    p = wl.paper_dataset(2, room=1, walls="eyring")
    assert p[0]["beta"][0] == wl.eyring_beta(wl.PAPER_ROOMS[1][0], wl.PAPER_RT)
