"""Plain, slow CPU oracle for the Pencil HE linear-layer hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import, call or execute it.  It
shares no code, header, table or constant generator with the CUDA library in
``paper_2403_11166_gb300/``; the two meet only in the seeded input generators
(``paper_2403_11166_gb300/inputs.py``), which hold none of the method's
arithmetic.

Everything here is written from the paper (Pencil, NDSS 2024) and from the
textbook definitions it relies on:

* ``params``   -- BFV parameters {N, t, q} with RNS primes (Sec. 2.2, Sec. 5
                  "RNS Decomposition").
* ``philox``   -- Philox4x64-10 counter-based generator (Salmon et al., SC'11),
                  the randomness source for keys, encryption, masks.
* ``sampling`` -- ternary secret, uniform-mod-q, discrete-Gaussian (CDT),
                  uniform Z_t masks drawn from fixed Philox streams.
* ``ntt``      -- negacyclic NTT by its definition (O(N^2)) and by a plain
                  radix-2 loop (Sec. 5 "NTT").
* ``ring``     -- schoolbook negacyclic product, direct ring matmul / conv.
* ``bfv``      -- symmetric BFV keygen / encrypt / add_plain / mul_plain /
                  decrypt with exact big-integer CRT (Sec. 2.2).
* ``packing``  -- polynomial encodings pi_v, pi_W, pi_y^{-1} (Appendix A) and
                  a brute-force collision checker.
* ``protocol`` -- Algorithm 1 (forward), the Algorithm-1-like grad_X step and
                  Algorithm 2 (grad_W cross terms) over shares.

Functions whose correctness has no independent pin say "parity unpinned" in
their docstring.  All current functions are pinned by ``tests/test_oracle_*``.
"""
