"""CPU oracle for the footprint-NDF / CP range-query path (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes anything here, and this
package imports nothing from the product path: the two share only the seeded
input generators in ``synth``.

Everything is plain numpy in FP64 (integers in int64), written from the paper
(Constant-Cost Spatio-Angular Prefiltering of Glinty Appearance Using Tensor
Decomposition, arXiv 2109.14807):

* ``ndf``   -- normal binning and exhaustive multi-level footprint histograms
               (Sec. 4.1), the normalised NDF tensor;
* ``cp``    -- CP decomposition by alternating least squares (Sec. 4.2, Eq. 3),
               with the MTTKRP on the dense tensor, streamed level by level,
               or in the structured form that moves the footprint window onto
               the spatial factors (exact, O(N^2 L R));
* ``query`` -- point query (Sec. 4.3, Eq. 4), range query through 1D summed-area
               tables (Sec. 4.4, Eq. 5 and the Appendix proposition), the dense
               brute-force range average it must equal, and the adjoint of the
               range query.

* ``clustered`` -- the clustered compression layout of Sec. 4.2 (t x t angular
               blocks, 8 x 8-texel regions, blank blocks dropped, a 3-mode CP
               per group) and its block-splitting range query (Sec. 4.4);
* ``sampling`` -- hierarchical NDF importance sampling (Sec. 5.2).

Parity pins (what fixes each function to something other than itself) live in
``tests/test_oracle_*.py``.  No function here is "parity unpinned".
"""
from . import ndf, cp, query, clustered, sampling  # noqa: F401
