"""Host-side checks of the many-mock batch recipe and of the batch ABI's
argument handling (no GPU)."""
import numpy as np

from paper_1705_03464_gb300 import synth


def test_many_mocks_recipe():
    mocks = synth.many_mocks(64)
    assert len(mocks) == 64
    Ls = np.array([w.box_L for w, _ in mocks])
    Ns = np.array([w.mesh_n for w, _ in mocks])
    ng = np.array([w.n_gal for w, _ in mocks])
    assert Ls.min() >= 256 and Ls.max() <= 1100
    assert set(Ns) <= {256, 512, 1024} and len(set(Ns)) == 3
    # cells of about 1 Mpc/h: the nearest power of two to L
    for L, N in zip(Ls, Ns):
        assert N == 2 ** int(np.clip(np.round(np.log2(L)), 8, 10))
    assert ng.min() >= 2e4 and ng.max() <= 4e5
    for w, hod in mocks:
        assert abs(hod[0] - synth.HOD_Z09[0]) <= 0.2 and abs(hod[1] - synth.HOD_Z09[1]) <= 0.2
        for k in (2, 3, 4):
            assert abs(np.log10(hod[k] / synth.HOD_Z09[k])) <= 0.2 + 1e-12
        assert len(w.s_edges) == 21 and w.n_mu == 5 and len(w.r_edges) == 11 and w.n_mur == 5
        assert w.r_edges[-1] < w.box_L / 2
    # deterministic in the seed
    again = synth.many_mocks(3)
    assert [w.box_L for w, _ in again] == list(Ls[:3])


def test_many_mocks_catalogue_size():
    w, hod = synth.many_mocks(1, seed0=5)[0]
    cat = synth.make_catalogue(w, 5, hod)
    assert abs(cat.n - w.n_gal) < 0.2 * w.n_gal
    assert cat.pos.min() >= 0 and cat.pos.max() < w.box_L
