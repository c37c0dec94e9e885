"""GB300 (sm_103a) library for the matrix-valued quantum Boltzmann equation of
Lu & Mendl (arXiv:1408.1782): fast spectral collision operator, minmod
transport, precession and the split time step, behind a C ABI."""
