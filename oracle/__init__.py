"""CPU oracle for the TNMH proposal path (test infrastructure only).

This package is a plain, slow, FP64 restatement of the method of
Frias-Perez et al., "Collective Monte Carlo updates through tensor network
renormalization" (arXiv:2104.13264).  It exists to check the CUDA path; only
the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
never calls into it and it shares no code with ``paper_2104_13264_gb300``.

Modules
-------
philox   Philox4x32-10 counter-based generator (Salmon et al., SC'11).
tnmc     boundary-MPS builder (App. A, eq. braket-top-tm-bot), sequential
         sampler / evaluator of the approximate prior (Sec. 2, eqs. bayes,
         pi-approx, tns-prior), Ising energy (eq. ising), MH scan (eq. mh-acc,
         Algorithm 1) and the reverse-mode gradient of log q.
exact    brute-force references used only to pin the oracle: enumeration of
         all states, row transfer matrix, Onsager free energy, the exact
         stationary acceptance of an independence sampler.
"""
