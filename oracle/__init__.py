"""Plain FP64 CPU oracle for the MQ-RBF Helmholtz Krylov-regularization path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The library (``paper_2511_09798_gb300``) never does,
and this package imports nothing from it: the two share no code.  Inputs come
from the separate ``workloads`` package, which holds no solver arithmetic.

Contents (each function cites the passage it follows):

* ``mq``         -- MQ basis Phi, Helmholtz operator L Phi, collocation matrix A
                    (Sec. 2.1, eqs. MQ, Lphi, H_entries, augmented_system).
* ``gkb``        -- Golub-Kahan bidiagonalization with full reorthogonalization
                    and breakdown halt (Algorithm 1, Sec. 3.1).
* ``regularize`` -- projected SVD, projected GCV and L-curve, Ine-TSVD, HKT,
                    full-SVD TSVD and Tikhonov with GCV (Algorithms 2-4,
                    eqs. tsvd_solution, tikh_svd_solution, rho, eta, gcv_svd,
                    rho_proj, eta_proj, gcv_proj).
* ``evaluate``   -- reconstruction u(X) and the relative error Re (eqs.
                    u_reconstruction, rel_error).
* ``mlp``        -- the stopping/lambda network's forward, backward and Adam
                    step (not in the paper; exact-erf GELU, Hendrycks & Gimpel;
                    Adam, Kingma & Ba).

All arithmetic is numpy float64.  Readings of passages where the paper is
silent or ambiguous are stated in each function's docstring.
"""
