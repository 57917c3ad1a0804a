// Instantiation of the CG solver for one (inner, accumulate, link compression, high) choice.
#include "dw_solver.cuh"
template struct dw::CG<dw::PI16, dw::P32, true, dw::PDF>;
