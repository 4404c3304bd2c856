"""GB300 (sm_103a) locally corrected quadrature: near-field correction generation for
Helmholtz layer potentials on curved triangular patches (arXiv 2006.02545).

  paper_2006_02545_gb300.lcq        ctypes binding of liblcq.so (the C ABI in include/lcq.h)
  paper_2006_02545_gb300.workloads  seeded synthetic surfaces, targets and densities
  paper_2006_02545_gb300.build      in-tree nvcc build of liblcq.so
"""
