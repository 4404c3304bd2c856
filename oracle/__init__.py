"""Plain FP64 CPU oracle for locally corrected quadrature corrections.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import or run anything in this package.  It shares no code
with the CUDA path (no kernels, headers, helpers, tables or table generators) and
never imports it.  Every function states the passage of Greengard, O'Neil, Rachh
and Vico, "Fast multipole methods for the evaluation of layer potentials with
locally-corrected quadratures" (arXiv 2006.02545), that it follows.

Two levels:
  * the scheme oracle (koornwinder, rules, geometry, kernels, nearlist, quadrature,
    corrections, apply): the discrete algorithm of Sec. 4-5 step by step, in the
    paper's order and notation, with the readings listed in the project's design
    notes where the paper is silent;
  * the truth oracle (truth): integrals to near machine precision by independent
    rules and closed forms, used to pin the scheme oracle.

Degrees: a degree-d patch has n = (d+1)(d+2)/2 nodes (paper order p = d+1).
"""
