"""CPU FP64 oracle for the coherent F-statistic template loop.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, step-by-step
restatement of the method in numpy float64.  Only the tests, the smoke check
and the CPU-baseline leg of the benchmark may import it; the library under
``paper_1003_0844_gb300`` never does, and this package imports nothing from
that library.

Modules and the parts of the paper they follow:

* ``earth``     analytic Earth: sky vector (Eq. pha4), detector position
                (Eq. pha5), the scalar product n0.r_d (Sec. II), site vector
                on the ellipsoid and Earth rotation (Sec. V); or a caller's
                table of the detector position and velocity on the sample grid
                (the ephemerides of Sec. V), read by linear extrapolation from
                the nearest grid point.
* ``response``  amplitude modulation functions a(t), b(t) (Sec. II; formulas
                of the cited interferometer response paper, Eqs. 12-13 there),
                the four-amplitude signal model (Eqs. sig, eq:ab, eq:ampone,
                h0iota) used to synthesise injections.
* ``resample``  barycentric source times (Eq. eq:Bt), Fourier x2 upsampling
                and natural cubic spline interpolation (Sec. VI.A).
* ``fstat``     Fa, Fb as transforms in barycentric time (Eq. ia), the DFT
                convention (Eq. eq:DFT), the F-statistic (Eq. OS), the exact
                F without resampling (Eqs. OS, Fab), threshold crossings, the
                noise-only false-alarm probability (Eq. PF).
* ``refine``    the fine search (Sec. VI.C): exact F at continuous points
                with its gradient, Hessian and reduced Fisher matrix (Eq.
                redFm-def), Nelder-Mead maximisation.
* ``adjoint``   the coarse search's F of the resampled series at continuous
                points and its gradient through the resampling (Eqs. eq:Bt,
                ia, Fab, OS; Sec. VI.A).
* ``grid``      the constrained A4* lattice covering (Sec. IV).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, a textbook/library special case or brute force, except the
readings the paper leaves open (spline end conditions, the Nyquist split of
the upsampler, the heterodyne reading, the edge rule of the resampler), whose
pins check only internal consistency: parity unpinned by the paper for those
readings.
"""
