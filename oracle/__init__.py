"""FP64 CPU oracle for the Split-SPCP hot path (Driggs, Becker, Aravkin, arXiv 1702.02241).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct NumPy
implementation of what the CUDA path computes.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product (``paper_1702_02241_gb300``) never imports it and shares no code with it; the one
shared module is the seeded input generator ``paper_1702_02241_gb300.gen``, which holds no
arithmetic of the method.

Modules and the passages they follow:

* ``core``        -- Huber value/derivative (Sec. 1 "Marginalization in S", Sec. 3.2), the
                     factored objective Eq. (Thm5) / Eq. (7) with the optional mask of Sec. 6.2,
                     its gradient (Sec. 3.2), the sparse part S.
* ``lbfgs``       -- L-BFGS with memory 10 (Sec. 5.1, Table 1) and a strong-Wolfe line search
                     (the paper is silent on the line search; Nocedal & Wright Alg. 3.5/3.6).
* ``certificate`` -- the convergence certificate of Sec. 3.4 (the four-term ||E||_F, the
                     QR + small-SVD route of its footnote, the distance bound F_bound).
* ``convex``      -- proximal gradient / FISTA with singular-value thresholding on Eq. (4)
                     (Sec. 1 notes proximal methods apply but need an SVD): reference solutions
                     on tiny instances; and the convex baseline of Sec. 6.1, the same iteration
                     with the thresholding done through a TSQR-based randomized SVD.
* ``tsqr``        -- TSQR, the QR of a tall-skinny matrix by a reduction tree of small QRs
                     (Sec. 6.1), normalised to a non-negative diagonal of R.
* ``sketch``      -- randomized-SVD initialisation U0 = U_k S^1/2, V0 = V_k S^1/2 (Sec. 4.2).
* ``quant``       -- the values X takes when stored as bfloat16 or FP8 E4M3 (per-column scale),
                     from the formats' definitions, for the precision form of the objective pass.
* ``frank_wolfe`` -- the Frank-Wolfe method with marginalization (Sec. 6.2, Algorithm 1): the
                     linear subproblem's top singular pair, the closed-form step, the gap.
* ``aicc``        -- the corrected Akaike information criterion of a solution (Sec. 5.2).
* ``warm_start``  -- the learned warm start (an extension: the paper compares SVD, rSVD and
                     random starts, Sec. 4.2): spectrum features of the sketch, the three-layer
                     network with bfloat16 weights, its gradient, Adam, the targets w*.

Every function is pinned by ``tests/test_oracle_*.py`` against something other than itself:
brute-force minimisation, finite differences, closed-form SVT solutions, the explicit
subdifferential construction, planted recovery.
"""
