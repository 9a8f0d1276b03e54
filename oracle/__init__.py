"""FP64 CPU oracle for the pair-galaxy cross-correlation (Yuan, Eisenstein &
Garrison 2017). TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct statement of what the GPU
path computes. Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the library itself never does, and it shares no code with the CUDA kernels.

Modules, each following the paper passage named in its docstring:

* ``pairs``     positions (wrap, RSD shift: Sec. 3.2 eq. RSD), direct O(N^2)
                pair enumeration binned by (s, mu) with pair midpoints
                (Sec. 2.1, eq. delta_pi_x), pair counts and xi(s, mu) = DD/RR - 1
                (Sec. 3.4, eq. 2PCF_d_collapsed).
* ``mesh``      NGP / CIC / TSC mass assignment in Q32.32 fixed point (Sec. 3.5).
* ``dft``       its own FP64 discrete Fourier transform (textbook
                Cooley-Tukey split over direct matrix DFTs).
* ``correlate`` the mesh cross-correlation C(r) (Sec. 2.1, eqs. bpg_initial,
                bpg_intermediate with a shell-indicator W), (r, mu_r) binning,
                b_pg, xi(d_w) (eq. xi_dw), Q_eff (eqs. Qeff, Qeff_notsq).
* ``direct``    the same correlation summed directly over (pair, galaxy)
                mesh-corner combinations (the triplet-counting form), used as a
                pin of ``correlate`` and for sampled checks at full size.
* ``pipeline``  the whole forward path for one catalogue.
* ``hod_grad``  soft HOD weights (Sec. 3.3 eq. hod) and reverse-mode
                gradients.

Parity unpinned: nothing here reproduces a number printed in the paper; the
paper's values need the Abacus simulations (Sec. 3.1), which are missing.
"""
