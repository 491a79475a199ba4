// Plan-specialised root pass: the code-generation layer of the engine (Fig. 1 of the paper
// compiles each optimised plan into code specialised for the batch). For a lean root pass
// (degree <= 2 basis over the root's value columns, at most one inner child) the shape of the
// batch -- monomials, inner view columns, histogram sets, root-to-inner columns, key domain --
// is turned into a CUDA kernel with straight-line per-tuple code and every constant folded,
// compiled at plan time with NVRTC for sm_103a and cached per process by its source text.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fastpass.cuh"

namespace lmfao {

struct GenRootPass {
  const void *fn = nullptr;  // kernel handle (cudaKernel_t) or null: the template kernel runs
  int block = 0;
  size_t smem = 0;
  std::string why;           // why the kernel was not generated (empty when it was)
};

// Generate (or take from the cache) the kernel for the lean root pass described by d.
// Returns a null handle, with the reason, when the shape is outside what is generated or
// when compilation fails; the caller then launches the template kernel.
GenRootPass gen_root_pass(const DFast &d, bool fp64, int device);

// Launch a generated root pass on stream s over `grid` CTAs.
cudaError_t launch_gen_root_pass(const GenRootPass &g, const DFast &d, int grid, cudaStream_t s);

// The source text that gen_root_pass compiles for d (for tests and inspection).
std::string gen_root_pass_source(const DFast &d, bool fp64, int block);

}  // namespace lmfao
