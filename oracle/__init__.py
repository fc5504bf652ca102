"""FP64 CPU oracle for the Pointing SelfCal hot path (test infrastructure).

This package is test infrastructure only.  It is a plain, slow, obviously
correct CPU restatement of what the paper's method computes, written from the
paper (Bhatnagar & Cornwell 2017) in double precision:

* ``model_grid``   -- V° = F[I^M], the model grid (Algorithm 1, first pre-compute)
* ``aperture``     -- A°, the a-priori aperture kernel, and its radial table
                      (Algorithm 1, second pre-compute; Sec. 3)
* ``degrid``       -- per-visibility sums with the pointing-modified kernel
                      A_ij (Eq. AIJPOINTING) and its derivative (Eq. DAIJPOINTING)
* ``psc``          -- model visibilities, derivatives, residuals, chi^2 and the
                      per-antenna gradient and 2x2 normal blocks (Eqs. Chisq, DCHIDD)
* ``closed_form``  -- direct-sum visibilities of point sources under shifted
                      primary beams (Eq. ME; the paper's simulation, Sec. 4.1)
* ``lm``           -- Levenberg-Marquardt minimiser standing in for the
                      paper's unspecified f() and Terminate() (Sec. 2.2, Algorithm 1)
* ``exact``        -- the exact kernel of two shifted uniform-disk patterns
                      (Sec. 3's more accurate pattern), quadrature in ``exact.c``
* ``wsnap``        -- W-snapshots: the interval's least-squares uvw plane and
                      the sky moved to the snapshot frame (Sec. 6.1)
* ``wstack``       -- what W-snapshots leave on long intervals: the model grid
                      stacked in the residual w, interpolated per visibility

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The GPU library shares no code with it.
"""
