"""Pins of the oracle's mass assignment and its own DFT."""
import numpy as np
import pytest

from oracle import dft, mesh as om

TWO32 = 2 ** 32


def test_ngp_is_a_histogram():
    L, N = 32.0, 16
    rng = np.random.default_rng(0)
    p = rng.random((500, 3)) * L
    m = om.deposit(p, None, L, N, 0)
    # textbook NGP: count of points whose nearest node (periodic) is each node
    node = np.floor(p / (L / N) + 0.5).astype(int) % N
    h, _ = np.histogramdd(node[:, ::-1], bins=(N, N, N), range=((0, N),) * 3)
    assert np.array_equal(m, h.astype(np.int64) * TWO32)


def test_cic_point_on_node_and_mass():
    L, N = 32.0, 16
    dx = L / N
    m = om.deposit(np.array([[3 * dx, 5 * dx, 7 * dx]]), np.array([0.5]), L, N, 1)
    assert m[7, 5, 3] == TWO32 // 2 and np.count_nonzero(m) == 1
    rng = np.random.default_rng(1)
    p = rng.random((400, 3)) * L
    w = rng.random(400)
    mm = om.deposit(p, w, L, N, 1)
    # total mass: exact up to one rounding (<= 1/2) per corner
    assert abs(int(mm.sum()) - float(np.sum(w) * TWO32)) <= 4 * 400
    # CIC preserves the centre of mass of a point away from the boundary
    q = np.array([[10.3, 11.7, 12.2]])
    mq = om.deposit(q, None, L, N, 1)
    idx = np.nonzero(mq)
    com = [np.sum(mq[idx] * idx[k]) / TWO32 * dx for k in range(3)]
    assert np.allclose(com[::-1], q[0], atol=1e-8)


def test_cic_wraps_periodically():
    L, N = 16.0, 8
    dx = L / N
    m = om.deposit(np.array([[L - 0.5 * dx, 0.0, 0.0]]), None, L, N, 1)
    assert m[0, 0, N - 1] == TWO32 // 2 and m[0, 0, 0] == TWO32 // 2


@pytest.mark.parametrize("n", [8, 12, 64, 128, 512, 1024])
def test_dft_matches_library_fft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((4, n)) + 1j * rng.standard_normal((4, n))
    for sign, ref in ((-1, np.fft.fft(x, axis=-1)), (+1, np.fft.ifft(x, axis=-1) * n)):
        y = dft.dft_last(x, sign)
        assert np.max(np.abs(y - ref)) < 1e-12 * np.max(np.abs(ref))


def test_dft3_against_definition_8cubed():
    rng = np.random.default_rng(3)
    n = 8
    x = rng.standard_normal((n, n, n))
    idx = np.indices((n, n, n)).reshape(3, -1)
    phase = np.exp(-2j * np.pi * (idx.T @ idx) / n)   # full M^2 DFT matrix
    ref = (phase @ x.reshape(-1)).reshape(n, n, n)
    assert np.max(np.abs(dft.dft3(x) - ref)) < 1e-11


def test_dft3_parseval_delta_planewave_roundtrip():
    n = 16
    rng = np.random.default_rng(4)
    x = rng.standard_normal((n, n, n))
    F = dft.dft3(x)
    assert np.isclose(np.sum(np.abs(F) ** 2), n ** 3 * np.sum(x * x), rtol=1e-12)
    d = np.zeros((n, n, n)); d[0, 0, 0] = 1.0
    assert np.allclose(dft.dft3(d), 1.0)
    kz, ky, kx = 3, 5, 1
    z, y, xx = np.indices((n, n, n))
    pw = np.exp(2j * np.pi * (kz * z + ky * y + kx * xx) / n)
    P = dft.dft3(pw)
    assert np.isclose(abs(P[kz, ky, kx]), n ** 3)
    P[kz, ky, kx] = 0
    assert np.max(np.abs(P)) < 1e-9
    back = dft.dft3(F, +1) / n ** 3
    assert np.max(np.abs(back - x)) < 1e-12
