"""CPU oracle for the transpose-algorithm multidimensional FFT (arXiv:1804.09536).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute anything in this package: only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
It shares no code with the CUDA path (no kernels, headers, helpers or tables)
and does not import the product package.

Plain, slow, obviously-correct NumPy in float64 / complex128:

* ``decomp``       -- balanced block-contiguous decomposition (Sec. 3.1, Eq. decompose,
                      Alg. 1), subarray boxes (Alg. 2), the virtual Cartesian process
                      grid and its one-dimensional subgroups (Sec. 3.4), and the stage
                      layouts of the slab / pencil / higher-dimensional methods
                      (Eqs. slab0-slab1, pencil0-pencil2, 4d_fft0-4d_fft3).
* ``redistribute`` -- index-level global redistribution: gather/scatter by slicing,
                      the subarray + all-to-all-w exchange (Alg. 3, Eq. gt), and the
                      traditional local transpose + all-to-all (Sec. 3.3.1, Eq. transpose).
* ``dft``          -- per-axis DFT as an exact-angle matrix product (Eqs. 1-2,
                      Eq. multifft), the forward / backward d-D transforms in the
                      paper's axis order (Eqs. fftn_forward / fftn_backward), the same
                      transforms run rank by rank on the virtual grid with exchanges in
                      between (Sec. 3.3-3.6), real-to-complex / complex-to-real
                      (footnote to Eq. multifft), and a brute-force full DFT.
* ``loss``         -- the spectral-weight loss sum |F(x) w|^2 and its gradient
                      2 F^H (w^2 F x), with F^H = (1/N) * backward.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or a library routine; none is
"parity unpinned".
"""
from . import decomp, redistribute, dft, loss  # noqa: F401
