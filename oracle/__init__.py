"""Plain FP64 CPU oracle for the nodal DG shallow-water method of arXiv:1403.1661.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` use it. It shares no code with the CUDA path (own reference element,
own rules, own connectivity, own right-hand side, own limiters, own multirate
integrator), and it is written for readability, not speed: every step follows
the paper's definitions in the paper's order, vectorised over elements with
numpy only where the same formula applies to every element.

Modules
-------
refelem   reference triangle: Warp & Blend nodes, orthonormal basis, cubature and
          Gauss rules, projection / interpolation / lift operators (Section 3).
mesh      connectivity, affine geometry, face point matching, CFL step and
          level grouping (Sections 3-4).
swe       fluxes, well-balanced Lax-Friedrichs flux, right-hand side (Sections 2,
          3, 5.1, 7.1, 7.2).
limiters  positivity-preserving limiter (Algorithm 3) and the characteristic TVB
          limiter with the positivity modification (Section 5.3).
mrab      multirate Adams-Bashforth integration with limiting (Algorithms 1, 2).

Parity status: every function is pinned by a test in tests/test_oracle_*.py
(closed forms, invariants, brute force); none is marked "parity unpinned".
"""
