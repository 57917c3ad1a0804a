// Instantiations of the CG solver for the covariant Laplacian: FP32 inner
// (18-real links) with IEEE FP64 or double-float corrections.
#include "dw_solver.cuh"
template struct dw::CG<dw::P32, dw::P32, false, dw::P64, dw::OP_LAPLACE>;
template struct dw::CG<dw::P32, dw::P32, false, dw::PDF, dw::OP_LAPLACE>;
