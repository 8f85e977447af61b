"""Plain, slow FP64 CPU oracle for the CLR (block-rank-sparse) product and the Newton–Schulz
S^-1/2 iteration of Calvin, Lewis & Valeev, "Scalable Task-Based Algorithm for Multiplication
of Block-Rank-Sparse Matrices" (IA^3 2015).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs may import this package.  The library
(``paper_1509_00309_gb300``) never imports it and shares no code with it: the only common
module is the seeded input generator ``paper_1509_00309_gb300.workloads``, which holds none of
the method's arithmetic.

Modules:
  clr_oracle    -- CLR representation, build (Section 4.1), product (Section 4.1 block
                   arithmetic + screening), linear combination, Newton–Schulz (Section 4.2),
                   the Daleckii–Krein gradient of trace(W S^-1/2) and the NS adjoint.
  split_oracle  -- bit-level bfloat16 rounding and the exact value of a split-precision
                   (multi-term bf16) product, used to check split tensor-core products.
  ozaki_oracle  -- exact-slice (Ozaki-scheme) digits, exponents and the exact value of the
                   sliced product, used to check the FP64-accurate tensor-core products.
"""
