// Instantiation of the CG solver for the covariant Laplacian: IEEE FP64 throughout.
#include "dw_solver.cuh"
template struct dw::CG<dw::P64, dw::P64, false, dw::P64, dw::OP_LAPLACE>;
