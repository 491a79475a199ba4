// Projection combine (see DComb4 in kernels.cuh).
//
//   tab_kernel      the outer terms and cells of each entry class, once per value of the
//                   class's digit(s) (view rows looked up by those digits alone);
//   proj_d0_kernel  one thread per Y column, one major digit and a chunk of minor digits per
//                   CTA: Yd0[d0][c] = SUM_d1 Y_c(d0, d1), and the column totals;
//   proj_d1_kernel  one thread per Y column, one minor digit (and a range of major digits)
//                   per CTA: Yd1[d1][c] = SUM_d0 Y_c(d0, d1);
//   class3_kernel   one thread per entry that needs every segment, a range of segments per
//                   CTA, summed per cell in shared memory;
//   entry_kernel    one warp per class 0..2 entry: tabulated term x projection per value of
//                   its digit, summed per cell in shared memory, then written out.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace lmfao {

namespace {


__device__ __forceinline__ bool cmp4(double x, double t, int op) {
  switch (op) {
    case LMFAO_LE: return x <= t;
    case LMFAO_LT: return x < t;
    case LMFAO_GE: return x >= t;
    case LMFAO_GT: return x > t;
    case LMFAO_EQ: return x == t;
    default: return x != t;
  }
}

// row of outer view o at digits (d0, d1)
__device__ __forceinline__ long long okey(const DComb2 &d, int o, int64_t d0, int64_t d1) {
  return d0 * d.outer[o].dstride[0] + d1 * d.outer[o].dstride[1];
}

// outer term t at digits (d0, d1), in FP64 (and exactly, when the term is integral); with
// skip0 the COUNT columns (column 0) of the outer views are taken as 1
__device__ void psi_at(const DComb2 &d, int t, int64_t d0, int64_t d1, double &v, unsigned long long &iv,
                       bool skip0) {
  const DPsi p = d.psi[t];
  v = 1.0;
  iv = 1ull;
  for (int f = p.f0; f < p.f0 + p.nf; ++f) {
    const DSegFac q = d.segfacs[f];
    const int64_t dg = q.digit == 0 ? d0 : d1;
    if (q.ind) {
      if (!cmp4((double)dg, (double)q.t, q.op)) { v = 0.0; iv = 0ull; }
    } else {
      double y = 1.0;
      unsigned long long iy = 1ull;
      for (int e = 0; e < q.pow; ++e) { y *= (double)dg; iy *= (unsigned long long)dg; }
      v *= y;
      iv *= iy;
    }
  }
  for (int i = p.p0; i < p.p0 + p.np; ++i) {
    const int2 sc = d.stage_col[d.psi_stage[i]];
    if (skip0 && sc.y == 0) continue;
    const double x = __ldg(d.outer[sc.x].v.v64 + okey(d, sc.x, d0, d1) * d.outer[sc.x].v.ncols + sc.y);
    v *= x;
    iv *= (unsigned long long)x;
  }
  if (!p.integral) iv = 0ull;
}

// outer cell of set og at digits (d0, d1): the query cell (cstride null) or the compact index
// over the set's own attributes; -1 when a code is missing
__device__ long long cell_at(const DComb2 &d, int og, int64_t d0, int64_t d1, const long long *cstride) {
  long long cell = 0;
  for (int r = d.og_off[og]; r < d.og_off[og + 1]; ++r) {
    const DGroupRef q = d.grefs[r];
    long long code;
    if (q.src == 0) code = q.a == 0 ? d0 : d1;
    else code = __ldg(d.outer[q.a].v.codes + okey(d, q.a, d0, d1) * d.outer[q.a].v.ncodes + q.b);
    if (code < 0) return -1;
    cell += code * (cstride ? cstride[r] : q.stride);
  }
  return cell;
}

template <typename T>
__device__ __forceinline__ double yflt(const DComb2 &d, int64_t s, int col) {
  return col < d.n0f ? (double)reinterpret_cast<const T *>(d.phi0f)[s * d.n0f + col]
                     : (double)d.phi1f[s * d.phi1f_seg + (col - d.n0f)];
}
__device__ __forceinline__ unsigned long long yint(const DComb2 &d, int64_t s, int col) {
  return col < d.n0i ? d.phi0i[s * d.n0i + col] : (unsigned long long)d.phi1i[s * d.phi1i_seg + (col - d.n0i)];
}

// Y_c(s) on a live segment, 0 elsewhere (the load does not depend on the liveness test, so
// the loads of an unrolled loop are all in flight together)
template <typename T>
__device__ __forceinline__ void yat(const DComb2 &d, int64_t s, int2 jb, double &yf, unsigned long long &yi) {
  const bool live = d.wseg[s] != 0ull;
  if (jb.x) {
    const unsigned long long y = yint(d, s, jb.y);
    yi = live ? y : 0ull;
    yf = 0.0;
  } else {
    const double y = yflt<T>(d, s, jb.y);
    yf = live ? y : 0.0;
    yi = 0ull;
  }
}

// grid (dom0, column tiles, chunks of the minor digit)
template <typename T>
__global__ void __launch_bounds__(256) proj_d0_kernel(const DComb4 dp) {
  const DComb2 &d = dp.c;
  const int J = blockIdx.y * blockDim.x + threadIdx.x;
  if (J >= dp.njobs) return;
  const int2 jb = dp.job[J];
  const int m = dp.dom1;
  const int64_t d0 = blockIdx.x;
  const int per = (m + gridDim.z - 1) / gridDim.z;
  const int a = blockIdx.z * per, b = min(m, a + per);
  double sf = 0.0;
  unsigned long long si = 0ull;
#pragma unroll 8
  for (int v = a; v < b; ++v) {
    double yf;
    unsigned long long yi;
    yat<T>(d, d0 * m + v, jb, yf, yi);
    sf += yf;
    si += yi;
  }
  if (jb.x) {
    if (si) {
      if (dp.need_d0) atomicAdd(dp.yd0_i + d0 * dp.njobs + J, si);
      atomicAdd(dp.yall_i + J, si);
    }
  } else if (sf != 0.0) {
    if (dp.need_d0) atomicAdd(dp.yd0_f + d0 * dp.njobs + J, sf);
    atomicAdd(dp.yall_f + J, sf);
  }
}

// terms and cells of entry class cls at every value of its digit(s)
__global__ void tab_kernel(const DComb4 dp, int cls) {
  const DComb2 &d = dp.c;
  const DTab4 &tb = dp.tab[cls];
  const int w = tb.nt + tb.ng;
  const int64_t nv = cls == 1 ? dp.dom0 : cls == 2 ? dp.dom1 : d.nseg;
  const int64_t n = nv * w;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i / w;
    const int k = (int)(i - x * w);
    int64_t d0 = 0, d1 = 0;
    if (cls == 1) d0 = x;
    else if (cls == 2) d1 = x;
    else { d0 = x / dp.dom1; d1 = x - d0 * dp.dom1; }
    const bool live = cls != 3 || d.wseg[x] != 0ull;
    if (k < tb.nt) {
      double v = 0.0;
      unsigned long long iv = 0ull;
      if (live) psi_at(d, tb.t[k], d0, d1, v, iv, dp.skip_counts != 0);
      tb.pf[x * tb.nt + k] = v;
      tb.pi[x * tb.nt + k] = iv;
    } else {
      tb.cell[x * tb.ng + (k - tb.nt)] =
          live ? cell_at(d, tb.g[k - tb.nt], d0, d1, dp.og_cstride) : -1;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) proj_d1_kernel(const DComb4 dp) {
  const DComb2 &d = dp.c;
  const int J = blockIdx.y * blockDim.x + threadIdx.x;
  if (J >= dp.njobs) return;
  const int2 jb = dp.job[J];
  const int m = dp.dom1, v = blockIdx.x;
  const int64_t per = (dp.dom0 + gridDim.z - 1) / gridDim.z;
  const int64_t a = (int64_t)blockIdx.z * per, b = min((int64_t)dp.dom0, a + per);
  double sf = 0.0;
  unsigned long long si = 0ull;
  if (dp.need_d1) {
#pragma unroll 8
    for (int64_t d0 = a; d0 < b; ++d0) {
      double yf;
      unsigned long long yi;
      yat<T>(d, d0 * m + v, jb, yf, yi);
      sf += yf;
      si += yi;
    }
  }
  if (dp.need_d1) {
    if (jb.x) { if (si) atomicAdd(dp.yd1_i + (int64_t)v * dp.njobs + J, si); }
    else if (sf != 0.0) atomicAdd(dp.yd1_f + (int64_t)v * dp.njobs + J, sf);
  }
}

// class 3 entries: grid (segment ranges, entry tiles), one thread per entry; an entry sums
// into its own cells in shared memory without atomics, written out once per CTA
template <typename T>
__global__ void __launch_bounds__(256) class3_kernel(const DComb4 dp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DComb2 &d = dp.c;
  double *sf = reinterpret_cast<double *>(smem);
  unsigned long long *si = reinterpret_cast<unsigned long long *>(smem);
  for (int i = threadIdx.x; i < dp.max_slots3; i += blockDim.x) si[i] = 0ull;
  __syncthreads();
  const int ei = blockIdx.y * blockDim.x + threadIdx.x;
  if (ei >= dp.nent3) return;  // no CTA-wide barrier follows
  const DEntry4 e = dp.ent3[ei];
  const int2 jb = dp.job[e.job];
  const DTab4 &tb = dp.tab[3];
  const int64_t per = (d.nseg + gridDim.x - 1) / gridDim.x;
  const int64_t a = (int64_t)blockIdx.x * per, b = min(d.nseg, a + per);
  constexpr int U = 4;  // segments whose loads are issued together
  for (int64_t s0 = a; s0 < b; s0 += U) {
    long long cl[U];
    double pf[U], yf[U];
    unsigned long long pi[U], yi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t s = s0 + u;
      const bool in = s < b;
      cl[u] = in ? tb.cell[s * tb.ng + e.tog] : -1;  // -1 also where w_s = 0
      pf[u] = in ? tb.pf[s * tb.nt + e.psi] : 0.0;
      pi[u] = in ? tb.pi[s * tb.nt + e.psi] : 0ull;
      yi[u] = in && jb.x ? yint(d, s, jb.y) : 0ull;
      yf[u] = in && !jb.x ? yflt<T>(d, s, jb.y) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (cl[u] < 0) continue;
      if (e.flags & 1) si[e.sbase + cl[u]] += pi[u] * yi[u];
      else sf[e.sbase + cl[u]] += pf[u] * (jb.x ? (double)yi[u] : yf[u]);
    }
  }
  const long long ncell = dp.og_ncells[e.og];
  const int r0 = d.og_off[e.og], r1 = d.og_off[e.og + 1];
  for (long long c = 0; c < ncell; ++c) {
    long long g = 0;
    for (int r = r0; r < r1; ++r) g += ((c / dp.og_cstride[r]) % dp.og_dom[r]) * d.grefs[r].stride;
    const long long idx = e.out + (g + e.icell) * e.cellmul;
    if (e.flags & 1) { if (si[e.sbase + c]) atomicAdd(d.icnt + idx, si[e.sbase + c]); }
    else if (sf[e.sbase + c] != 0.0) atomicAdd(d.fsum + idx, sf[e.sbase + c]);
  }
}

// one warp per class 0..2 entry; its cells in a per-warp region of shared memory
__global__ void __launch_bounds__(256) entry_kernel(const DComb4 dp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DComb2 &d = dp.c;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ei = blockIdx.x * (blockDim.x >> 5) + warp;
  if (ei >= dp.nent012) return;  // whole warps leave; no CTA-wide barrier follows
  const DEntry4 e = dp.ent[ei];
  double *sf = reinterpret_cast<double *>(smem) + (size_t)warp * dp.max_cells;
  unsigned long long *si = reinterpret_cast<unsigned long long *>(sf);
  const long long ncell = dp.og_ncells[e.og];
  const bool integ = (e.flags & 1) != 0, yint_col = (e.flags & 2) != 0;
  for (long long c = lane; c < ncell; c += 32) si[c] = 0ull;
  __syncwarp();
  const int J = e.job;
  const int n = e.cls == 0 ? 1 : e.cls == 1 ? dp.dom0 : dp.dom1;
  const DTab4 &tb = dp.tab[e.cls == 0 ? 1 : e.cls];
  for (int x = lane; x < n; x += 32) {
    double yf = 0.0;
    unsigned long long yi = 0ull;
    if (e.cls == 0) {
      if (yint_col) yi = dp.yall_i[J];
      else yf = dp.yall_f[J];
    } else {
      const int64_t at = (int64_t)x * dp.njobs + J;
      if (yint_col) yi = e.cls == 1 ? dp.yd0_i[at] : dp.yd1_i[at];
      else yf = e.cls == 1 ? dp.yd0_f[at] : dp.yd1_f[at];
    }
    if (yi == 0ull && yf == 0.0) continue;
    const long long cell = e.cls == 0 ? 0 : tb.cell[(int64_t)x * tb.ng + e.tog];
    if (cell < 0) continue;
    double pv = 1.0;
    unsigned long long pi = 1ull;
    if (e.cls != 0) {
      pv = tb.pf[(int64_t)x * tb.nt + e.psi];
      pi = tb.pi[(int64_t)x * tb.nt + e.psi];
    }
    if (integ) atomicAdd(si + cell, pi * yi);
    else atomicAdd(sf + cell, pv * (yint_col ? (double)yi : yf));
  }
  __syncwarp();
  const int r0 = d.og_off[e.og], r1 = d.og_off[e.og + 1];
  for (long long c = lane; c < ncell; c += 32) {
    long long g = 0;
    for (int r = r0; r < r1; ++r) g += ((c / dp.og_cstride[r]) % dp.og_dom[r]) * d.grefs[r].stride;
    const long long idx = e.out + (g + e.icell) * e.cellmul;
    if (integ) { if (si[c]) atomicAdd(d.icnt + idx, si[c]); }
    else if (sf[c] != 0.0) atomicAdd(d.fsum + idx, sf[c]);
  }
}

}  // namespace

void launch_combine4(const DComb4 &d, bool fp64, cudaStream_t s) {
  const int bs = 256;
  const int tiles = (d.njobs + bs - 1) / bs;
  for (int cls = 1; cls <= 3; ++cls) {
    const int64_t nv = cls == 1 ? d.dom0 : cls == 2 ? d.dom1 : d.c.nseg;
    const int64_t n = nv * (int64_t)(d.tab[cls].nt + d.tab[cls].ng);
    if (n) tab_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 148 * 8), 256, 0, s>>>(d, cls);
  }
  // about four CTAs per SM in each projection
  const int z0 = std::max(1, std::min(d.dom1, (4 * 148 + d.dom0 * tiles - 1) / (d.dom0 * tiles)));
  if (fp64) proj_d0_kernel<double><<<dim3(d.dom0, tiles, z0), bs, 0, s>>>(d);
  else proj_d0_kernel<float><<<dim3(d.dom0, tiles, z0), bs, 0, s>>>(d);
  if (d.nent3) {
    const int etiles = (d.nent3 + bs - 1) / bs;
    const int r3 = std::max(1, (2 * 148 + etiles - 1) / etiles);
    const size_t sm3 = (size_t)8 * std::max(1, d.max_slots3);
    if (fp64) {
      cudaFuncSetAttribute(class3_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
      class3_kernel<double><<<dim3(r3, etiles), bs, sm3, s>>>(d);
    } else {
      cudaFuncSetAttribute(class3_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
      class3_kernel<float><<<dim3(r3, etiles), bs, sm3, s>>>(d);
    }
  }
  if (d.need_d1) {
    const int z = std::max(1, std::min(d.dom0, (4 * 148 + d.dom1 * tiles - 1) / (d.dom1 * tiles)));
    if (fp64) proj_d1_kernel<double><<<dim3(d.dom1, tiles, z), bs, 0, s>>>(d);
    else proj_d1_kernel<float><<<dim3(d.dom1, tiles, z), bs, 0, s>>>(d);
  }
  if (d.nent012) {
    const int wpb = std::max(1, std::min(8, (int)(48 * 1024 / (8 * std::max(1, d.max_cells)))));
    entry_kernel<<<(d.nent012 + wpb - 1) / wpb, 32 * wpb, (size_t)8 * wpb * std::max(1, d.max_cells), s>>>(d);
  }
}

}  // namespace lmfao
