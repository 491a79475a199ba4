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
      if (dp.need_d0) atomicAdd(dp.yd0_i + (int64_t)J * dp.dom0 + d0, si);
      atomicAdd(dp.yall_i + J, si);
    }
  } else if (sf != 0.0) {
    if (dp.need_d0) atomicAdd(dp.yd0_f + (int64_t)J * dp.dom0 + d0, sf);
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
      const int64_t at = cls == 3 ? x * tb.nt + k : k * nv + x;  // classes 1, 2: by term, then digit
      tb.pf[at] = v;
      tb.pi[at] = iv;
    } else {
      tb.cell[cls == 3 ? x * tb.ng + (k - tb.nt) : (k - tb.nt) * nv + x] =
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
    if (jb.x) { if (si) atomicAdd(dp.yd1_i + (int64_t)J * dp.dom1 + v, si); }
    else if (sf != 0.0) atomicAdd(dp.yd1_f + (int64_t)J * dp.dom1 + v, sf);
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
  if (e.cls == 0) {
    if (lane == 0) {
      const unsigned long long yi = yint_col ? dp.yall_i[J] : 0ull;
      const double yf = yint_col ? 0.0 : dp.yall_f[J];
      if (integ) si[0] += yi;
      else sf[0] += yint_col ? (double)yi : yf;
    }
  } else {
    const unsigned long long *ypi = e.cls == 1 ? dp.yd0_i : dp.yd1_i;
    const double *ypf = e.cls == 1 ? dp.yd0_f : dp.yd1_f;
    // one cell (an ungrouped aggregate): lane sums in registers, one warp reduction, instead of
    // every lane adding to the same shared word
    unsigned long long li = 0ull;
    double lf = 0.0;
    const bool one = ncell == 1;
    constexpr int U = 4;  // digit values per lane whose loads are issued together
    for (int x0 = lane; x0 < n; x0 += 32 * U) {
      double yf[U], pv[U];
      unsigned long long yi[U], pi[U];
      long long cl[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int x = x0 + 32 * u;
        const bool in = x < n;
        const int64_t at = (int64_t)J * n + x;
        yi[u] = in && yint_col ? ypi[at] : 0ull;
        yf[u] = in && !yint_col ? ypf[at] : 0.0;
        cl[u] = in ? tb.cell[(int64_t)e.tog * n + x] : -1;
        pv[u] = in ? tb.pf[(int64_t)e.psi * n + x] : 0.0;
        pi[u] = in ? tb.pi[(int64_t)e.psi * n + x] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if ((yi[u] == 0ull && yf[u] == 0.0) || cl[u] < 0) continue;
        if (one) {
          if (integ) li += pi[u] * yi[u];
          else lf += pv[u] * (yint_col ? (double)yi[u] : yf[u]);
        } else if (integ) {
          atomicAdd(si + cl[u], pi[u] * yi[u]);
        } else {
          atomicAdd(sf + cl[u], pv[u] * (yint_col ? (double)yi[u] : yf[u]));
        }
      }
    }
    if (one) {
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        li += __shfl_xor_sync(0xffffffffu, li, o);
        lf += __shfl_xor_sync(0xffffffffu, lf, o);
      }
      if (lane == 0) {
        if (integ) si[0] += li;
        else sf[0] += lf;
      }
    }
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


// ------------------------------------------------------------------ streaming form
// CTA (x, y) covers the minor digits [x c1, x c1 + c1) and the major digits [y c0, y c0 + c0).
// Per major digit it stages the tile row's per-segment sums (a warp per segment, lanes over
// the jobs: coalesced), adds them to the CTA's minor-digit sums (each element by the thread
// that staged it), writes the row's major-digit partial, and lets each class 3 entry (one per
// thread) add the row's terms x sums into its cells. Every per-segment sum is read once.
template <typename T>
__global__ void proj_stream_kernel(const DComb4 dp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const DComb2 &d = dp.c;
  const int nj = dp.njobs, c1 = dp.c1;
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
  const DTab4 &tb = dp.tab[3];
  const int nt3 = dp.fused3 ? tb.nt : 0, ng3 = dp.fused3 ? tb.ng : 0;
  unsigned long long *stage = reinterpret_cast<unsigned long long *>(smem);
  unsigned long long *acc1 = stage + (size_t)c1 * nj;
  unsigned long long *slots = acc1 + (size_t)c1 * nj;
  double *tpf = reinterpret_cast<double *>(slots + (dp.fused3 ? dp.nslots3 : 0));  // the row's class 3 terms
  unsigned long long *tpi = reinterpret_cast<unsigned long long *>(tpf + (size_t)c1 * nt3);
  long long *tcl = reinterpret_cast<long long *>(tpi + (size_t)c1 * nt3);            // and cells
  int2 *sjob = reinterpret_cast<int2 *>(tcl + (size_t)c1 * ng3);                     // job descriptors
  for (int J = tid; J < nj; J += bs) sjob[J] = dp.job[J];
  const int x0 = blockIdx.x * c1, xn = min(c1, dp.dom1 - x0);
  const int y0 = blockIdx.y * dp.c0, y1 = min(dp.dom0, y0 + dp.c0);
  for (int i = tid; i < c1 * nj; i += bs) acc1[i] = 0ull;
  if (dp.fused3)
    for (int i = tid; i < dp.nslots3; i += bs) slots[i] = 0ull;
  DEntry4 e{};
  int2 ejb = make_int2(0, 0);
  const bool has_e = dp.fused3 && tid < dp.nent3;
  if (has_e) {
    e = dp.ent3[tid];
    ejb = dp.job[e.job];
  }
  __syncthreads();  // sjob
  for (int d0 = y0; d0 < y1; ++d0) {
    __syncthreads();  // the previous row's readers are done with stage
    for (int r = warp; r < xn; r += nwarp) {
      const int64_t s = (int64_t)d0 * dp.dom1 + x0 + r;
      const bool live = d.wseg[s] != 0ull;
#pragma unroll 4
      for (int J = lane; J < nj; J += 32) {
        const int2 jb = sjob[J];
        unsigned long long w = 0ull;
        if (jb.x) {
          const unsigned long long y = live ? yint(d, s, jb.y) : 0ull;
          w = y;
          acc1[r * nj + J] += y;
        } else {
          const double y = live ? yflt<T>(d, s, jb.y) : 0.0;
          w = (unsigned long long)__double_as_longlong(y);
          acc1[r * nj + J] = (unsigned long long)__double_as_longlong(__longlong_as_double((long long)acc1[r * nj + J]) + y);
        }
        stage[r * nj + J] = w;
      }
      for (int t = lane; t < nt3; t += 32) {
        tpf[r * nt3 + t] = tb.pf[s * tb.nt + t];
        tpi[r * nt3 + t] = tb.pi[s * tb.nt + t];
      }
      for (int g = lane; g < ng3; g += 32) tcl[r * ng3 + g] = tb.cell[s * tb.ng + g];
    }
    __syncthreads();
    // the row's major-digit partial
    for (int J = tid; J < nj; J += bs) {
      const int2 jb = sjob[J];
      unsigned long long si = 0ull;
      double sf = 0.0;
      for (int r = 0; r < xn; ++r) {
        const unsigned long long w = stage[r * nj + J];
        if (jb.x) si += w;
        else sf += __longlong_as_double((long long)w);
      }
      dp.yd0p[((size_t)blockIdx.x * dp.dom0 + d0) * nj + J] = jb.x ? si : (unsigned long long)__double_as_longlong(sf);
    }
    // class 3 entries of this thread
    if (has_e) {
      for (int r = 0; r < xn; ++r) {
        const long long cl = tcl[r * ng3 + e.tog];  // -1 also where w_s = 0
        if (cl < 0) continue;
        const unsigned long long w = stage[r * nj + e.job];
        if (e.flags & 1) {
          slots[e.pad + cl] += tpi[r * nt3 + e.psi] * (ejb.x ? w : 0ull);
        } else {
          const double y = ejb.x ? (double)w : __longlong_as_double((long long)w);
          const double v = tpf[r * nt3 + e.psi] * y;
          slots[e.pad + cl] = (unsigned long long)__double_as_longlong(__longlong_as_double((long long)slots[e.pad + cl]) + v);
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < xn * nj; i += bs) {
    const int r = i / nj, J = i - r * nj;
    dp.yd1p[((size_t)blockIdx.y * dp.dom1 + x0 + r) * nj + J] = acc1[i];
  }
  if (has_e) {
    const long long ncell = dp.og_ncells[e.og];
    const int r0 = d.og_off[e.og], r1 = d.og_off[e.og + 1];
    for (long long c = 0; c < ncell; ++c) {
      const unsigned long long w = slots[e.pad + c];
      if (!w) continue;
      long long g = 0;
      for (int r = r0; r < r1; ++r) g += ((c / dp.og_cstride[r]) % dp.og_dom[r]) * d.grefs[r].stride;
      const long long idx = e.out + (g + e.icell) * e.cellmul;
      if (e.flags & 1) atomicAdd(d.icnt + idx, w);
      else atomicAdd(d.fsum + idx, __longlong_as_double((long long)w));
    }
  }
}

// Sums of the partial projections: Yd0 (and the column totals) over the minor-digit tiles,
// Yd1 over the major-digit tiles.
__global__ void proj_reduce_kernel(const DComb4 dp) {
  const int nj = dp.njobs;
  const int64_t n0 = (int64_t)dp.dom0 * nj, n1 = dp.need_d1 ? (int64_t)dp.dom1 * nj : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n0 + n1; i += stride) {
    const bool one = i >= n0;
    const int64_t k = one ? i - n0 : i;
    const int J = (int)(k % nj);
    const int2 jb = dp.job[J];
    const int parts = one ? dp.ny : dp.nx;
    const int64_t pstride = (one ? (int64_t)dp.dom1 : (int64_t)dp.dom0) * nj;
    const unsigned long long *src = (one ? dp.yd1p : dp.yd0p) + k;
    unsigned long long si = 0ull;
    double sf = 0.0;
    for (int p = 0; p < parts; ++p) {
      const unsigned long long w = src[p * pstride];
      if (jb.x) si += w;
      else sf += __longlong_as_double((long long)w);
    }
    const int64_t dig = k / nj;
    if (one) {
      const int64_t at = (int64_t)J * dp.dom1 + dig;
      if (jb.x) dp.yd1_i[at] = si;
      else dp.yd1_f[at] = sf;
    } else {
      const int64_t at = (int64_t)J * dp.dom0 + dig;
      if (jb.x) {
        if (dp.need_d0) dp.yd0_i[at] = si;
        if (si) atomicAdd(dp.yall_i + J, si);
      } else {
        if (dp.need_d0) dp.yd0_f[at] = sf;
        if (sf != 0.0) atomicAdd(dp.yall_f + J, sf);
      }
    }
  }
}

}  // namespace

size_t combine4_stream_smem(const DComb4 &d) {
  const size_t t3 = d.fused3 ? (size_t)d.nslots3 + (size_t)d.c1 * (2 * d.tab[3].nt + d.tab[3].ng) : 0;
  return 8 * (2 * (size_t)d.c1 * d.njobs + t3 + (size_t)d.njobs);
}

void launch_combine4(const DComb4 &d, bool fp64, cudaStream_t s) {
  const int bs = 256;
  const int tiles = (d.njobs + bs - 1) / bs;
  for (int cls = 1; cls <= 3; ++cls) {
    const int64_t nv = cls == 1 ? d.dom0 : cls == 2 ? d.dom1 : d.c.nseg;
    const int64_t n = nv * (int64_t)(d.tab[cls].nt + d.tab[cls].ng);
    if (n) tab_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 148 * 8), 256, 0, s>>>(d, cls);
  }
  if (d.stream) {
    const size_t sm = combine4_stream_smem(d);
    const dim3 grid((unsigned)d.nx, (unsigned)d.ny);
    if (fp64) {
      cudaFuncSetAttribute(proj_stream_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      proj_stream_kernel<double><<<grid, d.sblock, sm, s>>>(d);
    } else {
      cudaFuncSetAttribute(proj_stream_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      proj_stream_kernel<float><<<grid, d.sblock, sm, s>>>(d);
    }
    const int64_t nred = (int64_t)d.dom0 * d.njobs + (d.need_d1 ? (int64_t)d.dom1 * d.njobs : 0);
    proj_reduce_kernel<<<(int)std::min<int64_t>((nred + 255) / 256, 148 * 8), 256, 0, s>>>(d);
    if (d.nent3 && !d.fused3) {
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
    if (d.nent012) {
      const int wpb = std::max(1, std::min(8, (int)(48 * 1024 / (8 * std::max(1, d.max_cells)))));
      entry_kernel<<<(d.nent012 + wpb - 1) / wpb, 32 * wpb, (size_t)8 * wpb * std::max(1, d.max_cells), s>>>(d);
    }
    return;
  }
  // about four CTAs per SM in each projection
  const int z0 = std::max(1, std::min(d.dom1, (4 * 148 + d.dom0 * tiles - 1) / (d.dom0 * tiles)));
  if (fp64) proj_d0_kernel<double><<<dim3(d.dom0, tiles, z0), bs, 0, s>>>(d);
  else proj_d0_kernel<float><<<dim3(d.dom0, tiles, z0), bs, 0, s>>>(d);
  if (d.nent3) {
    const int etiles = (d.nent3 + bs - 1) / bs;
    const int r3 = std::max(1, (6 * 148 + etiles - 1) / etiles);  // several CTAs per SM
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
