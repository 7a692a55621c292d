"""FP64 CPU oracle for the IRL linear-method hot path. TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (``bench.py --impl reference`` and the ``cpu_baseline`` field) may import
or run anything in this package. The product path never does: it fails loudly
when its CUDA library is missing.

The oracle is a plain, slow, obviously correct restatement of what the paper
defines (arXiv 2601.01437, Methods):

* ``og_rows.c``   per-row ln psi, O, E_loc, G and Slater-Condon connections
                  (plain C loops, FP64), driven through ``native``;
* ``fock``        sector enumeration and a brute-force Jordan-Wigner Fock-space
                  Hamiltonian used only to pin the Slater-Condon rules;
* ``lm``          weights, energy centring, explicit S~ and H~' (the linear
                  method's (p+1)x(p+1) matrices), the SHEP the paper solves
                  and the deflated GEVP it approximates;
* ``irl``         a plain CPU implicitly restarted Lanczos (Algorithms 1, 2).

It shares no code with the CUDA path; both take their inputs from ``synth``.
Parity of every function here is pinned by ``tests/test_oracle_*.py``
(brute force, finite differences, closed forms, library eigensolvers).
"""
from . import native, fock, lm, irl  # noqa: F401
