"""CPU oracle for the radiative hot path (view factors -> enforcement -> Gebhart REFs).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow, obviously correct
reference that the CUDA library is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` leg (and its
``--impl reference`` arm) may import it. It shares no code with
``paper_2511_04277_gb300`` and never imports it; the product path never imports
this package.

Modules (each function cites the passage of the thesis it follows):

* ``mcrt``       Monte Carlo ray tracing hit counts (Sec. 3.5.1, Eq. 3.15), plain C
                 compiled on first use (``mcrt.c``), brute force and a median-split BVH.
* ``enforce``    reciprocity (Eq. 3.20, 3.25), open-system closure (Eq. 3.36-3.40),
                 the iterative enforcer and the least-squares optimum with NNR and
                 SPVA (Sec. 3.5.5, App. A).
* ``multinode``  sub-surface -> surface -> node relations (Ch. 5, Eq. 5.28-5.29).
* ``gebhart``    REFs of closed and open systems (Eq. 4.5, B.1-B.11), steady radiative
                 balance (Eq. 3.13, 4.1-4.2), adjoint gradients and finite differences.

Floating point is fp64 throughout, except the ray geometry, which the ray
definition fixes to IEEE float32 with every operation rounded.
"""
