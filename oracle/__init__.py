"""CPU FP64 oracle of the Lyman-alpha pixel-pair estimator (arxiv 2507.00129).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may call it.  It shares no code, header, table or helper
with the CUDA library; both consume the seeded catalogues of
``paper_2507_00129_gb300.synth`` (which hold no estimator arithmetic).

Contents (each function cites the passage it follows):

* ``geometry``  -- unit vectors, half-angle cos/sin, (r_par, r_perp)  (Section 2.1)
* ``pairs``     -- the forest-pair set inside the angular cut        (Section 2.1)
* ``xi``        -- xi_A = sum w d w d / sum w w per bin, Eq. (2.4)
* ``project``   -- the continuum projection eta, Eq. (2.7)
* ``dmat``      -- distortion matrix D_AB, Eq. (2.6): literal and expanded forms
* ``subsample`` -- the seeded forest-pair subsample used for D    (Section 2.2)
* ``adjoint``   -- gradient of L = sum_A c_A xi_A w.r.t. delta and w (chain rule of Eq. 2.4)
* ``covariance``-- HEALPix sub-samples and the weighted sub-sample covariance of xi
* ``xi3``       -- the anisotropic three-point estimator, Eq. (2.8), on the 5-variable triangle grid
* ``xcf``       -- forest x quasar cross-correlation and its distortion matrix (readings of Eq. 2.4-2.7)
* ``xi1d``      -- the same-forest (1D) correlation that Eq. (2.4) excludes

Everything is float64.  Readings of passages the paper leaves open are listed
in the module docstrings.
"""
from . import geometry, pairs, xi, project, dmat, subsample, adjoint, covariance, xi3, xcf, xi1d  # noqa: F401
