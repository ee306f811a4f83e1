// Internal host interface between the time-loop drivers (aew_api.cu) and the
// optimisation drivers built on them (aew_newton.cu).  Not part of the public C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <string>

#include "../../include/aewave.h"

namespace aew {

struct GridInfo {
  int nx, ny, nz;
  double h;
  size_t C;   // nodes
};

GridInfo grid_of(const aew_handle* h);

// set the handle's error message; returns code
int set_error(aew_handle* h, int code, const std::string& msg);

// aew_gradient with an Armijo gate: once the forward solve has produced the misfit J,
// the call stops before the adjoint solve if J > gate (*accepted = false; g_dev is not
// written, the handle holds no gradient).  gate = +inf runs the whole gradient.  With
// revolve storage the misfit is known only at the end, so the gate is tested then.
// *misfit receives J either way.
int gradient_gated(aew_handle* h, const float* c_dev, const float* d_obs_dev, float* g_dev,
                   double gate, double* misfit, bool* accepted, cudaStream_t s);

}  // namespace aew
