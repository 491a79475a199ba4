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
  bool family = false;       // generated from the general shape (codegen_family.cpp)
  std::string why;           // why the kernel was not generated (empty when it was)
  std::string source_hash;   // FNV-1a (64-bit, hex) of the generated source: names the exact kernel
};

// Generate (or take from the cache) the kernel for the specialised root pass described by d:
// the lean generator for lean passes, the general one otherwise; thr are the host copies of
// the bucket thresholds the pass reads. Returns a null handle, with the reason, when the shape
// is outside what is generated or when compilation fails; the caller then launches the
// template kernel.
GenRootPass gen_root_pass(const DFast &d, bool fp64, int device, const std::vector<float> &thr);

// General shape (codegen_family.cpp): shared-memory layout, argument slots, eligibility
// and source.
struct FamilyLayout {
  int rs;
  int nfull, tew;  // FP32 rows: full 16-byte planes and the element width (words) of the tail plane
  bool pi_smem;  // integral root-to-inner partials in shared memory (also when the float ones are not)
  size_t off_tab, off_code, off_pf, off_pi, off_h, off_b4f, off_b4i, smem;
};
enum FamArg {
  F_NWORK, F_WORK, F_WSEG, F_WORKQ, F_TABLE, F_CODES, F_PHI0F, F_PHI0I, F_PHI1F, F_PHI1I, F_P3F, F_P3F32, F_P3I,
  F_FSUM, F_ICNT, F_KC, F_X0, F_OV0 = F_X0 + 6, F_NARGS = F_OV0 + 6
};
FamilyLayout family_layout(const DFast &d, bool fp64, int block);
bool family_eligible(const DFast &d, std::string &why, const std::vector<DGroupRef> &grefs4);
std::string gen_family_source(const DFast &d, bool fp64, int block, const std::vector<float> &thr,
                              const std::vector<DGroupRef> &grefs4, const std::vector<DMirror> &mirror);

// Launch a generated root pass on stream s over `grid` CTAs.
cudaError_t launch_gen_root_pass(const GenRootPass &g, const DFast &d, int grid, cudaStream_t s);

// Generated view kernel of a unique-key relation without children (codegen.cpp): the view's
// columns and codes as straight-line code per key; cfo, facs, cdesc and thr are the host copies
// of the kernel's column factor offsets, factors, code descriptors and bucket thresholds.
struct GenView {
  const void *fn = nullptr;  // null: view_key_rows_kernel runs
  std::string why, source_hash;
};
GenView gen_view(const DViewKernel &d, const std::vector<int> &cfo, const std::vector<DFac> &facs,
                 const std::vector<int4> &cdesc, const std::vector<float> &thr);
std::string gen_view_source(const DViewKernel &d, const std::vector<int> &cfo, const std::vector<DFac> &facs,
                            const std::vector<int4> &cdesc, const std::vector<float> &thr);
cudaError_t launch_gen_view(const GenView &g, const DViewKernel &d, cudaStream_t s);

// The source text that gen_root_pass compiles for d (for tests and inspection).
std::string gen_root_pass_source(const DFast &d, bool fp64, int block);

// Source of the warp's reduce-scatter of the V per-lane segment sums acc[0..V) of a work item
// into r_[]: with V <= 32, the values are padded to the next power of two PV = 2^L, reduced
// over L lane bits by exchanging halves (PV - 1 shuffles) and over the remaining 5 - L lane bits
// by butterflies, so that lane l holds value (l >> (5 - L)) in r_[0]; with V > 32, F = ceil(V / 32)
// values per lane, lane l holding values l F .. l F + F - 1 in r_[0..F).
struct WarpReduce {
  int V, F, shift;  // shift = 5 - L (V <= 32), else 0
  std::string src;
  // lane that holds value q (and the register it is in)
  int lane_of(int q) const { return F == 1 ? q << shift : q / F; }
  int reg_of(int q) const { return F == 1 ? 0 : q % F; }
};
WarpReduce gen_warp_reduce(int V, const std::string &ind);
// atomicAdd of every reduced value to dst[base + q] (the lane that owns it; zero values skipped)
std::string gen_reduce_flush(const WarpReduce &w, const std::string &dst, const std::string &base,
                             const std::string &ind);

}  // namespace lmfao
