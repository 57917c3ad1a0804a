// Instantiations of the CG solver for the covariant Laplacian: FP16 inner
// (12-real links) with IEEE FP64 or double-float corrections.
#include "dw_solver.cuh"
template struct dw::CG<dw::P16, dw::P32, true, dw::P64, dw::OP_LAPLACE>;
template struct dw::CG<dw::P16, dw::P32, true, dw::PDF, dw::OP_LAPLACE>;
