// CUDA kernels of the engine (sm_103a).
//
//  view_kernel        -- the view of a non-root relation r (Section 2): one pass over r per column,
//                        lookups into its children's views, accumulation of every needed
//                        product column per join key into a dense key-indexed array.
//  fact_pass          -- the root group (Section 2 multi-output plan; Fig. 3 loop nest with
//                        the segment key as outer level): one coalesced pass over the
//                        root relation, reorganised as segments; per tuple the inner view
//                        lookups and row terms; per segment the sums PHI (the view from
//                        the root to the segment relation); per tuple the direct items.
//  reorganisation     -- segment ids, histogram and scatter (plan time).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lmfao {

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ int ld_i32(const DCol &c, int64_t r) {
  return __ldg(reinterpret_cast<const int *>(c.p) + r);
}

template <typename T>
__device__ __forceinline__ T ld_num(const DCol &c, int64_t r) {
  if (c.dtype == LMFAO_F32) return (T)__ldg(reinterpret_cast<const float *>(c.p) + r);
  if (c.dtype == LMFAO_U8) return (T)__ldg(reinterpret_cast<const unsigned char *>(c.p) + r);
  return (T)__ldg(reinterpret_cast<const int *>(c.p) + r);
}

template <typename X>
__device__ __forceinline__ bool cmp_op(X x, X t, int op) {
  switch (op) {
    case LMFAO_LE: return x <= t;
    case LMFAO_LT: return x < t;
    case LMFAO_GE: return x >= t;
    case LMFAO_GT: return x > t;
    case LMFAO_EQ: return x == t;
    default: return x != t;
  }
}

// Predicates compare the stored value: FP32 columns in FP32, integer columns exactly.
__device__ __forceinline__ bool pred_at(const DCol &c, int64_t r, int op, float t) {
  if (c.dtype == LMFAO_F32) return cmp_op<float>(__ldg(reinterpret_cast<const float *>(c.p) + r), t, op);
  double x = (c.dtype == LMFAO_U8) ? (double)__ldg(reinterpret_cast<const unsigned char *>(c.p) + r)
                                   : (double)__ldg(reinterpret_cast<const int *>(c.p) + r);
  return cmp_op<double>(x, (double)t, op);
}

template <typename T>
__device__ __forceinline__ T fac_at(const DCol *cols, const DFac &f, int64_t r) {
  const DCol &c = cols[f.col];
  if (f.ind) return pred_at(c, r, f.op, f.t) ? T(1) : T(0);
  T x = ld_num<T>(c, r);
  T v = x;
  for (int p = 1; p < f.pow; ++p) v *= x;
  return v;
}

// bucket(x) = number of thresholds strictly below x
__device__ __forceinline__ int bucket_of(float x, const float *thr, int n) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(thr + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int code_at(const DCol &c, int64_t r, int kind, const float *thr, int nthr) {
  if (kind == LMFAO_GB_BUCKET) {
    float x = (c.dtype == LMFAO_F32) ? __ldg(reinterpret_cast<const float *>(c.p) + r)
              : (c.dtype == LMFAO_U8) ? (float)__ldg(reinterpret_cast<const unsigned char *>(c.p) + r)
                                      : (float)__ldg(reinterpret_cast<const int *>(c.p) + r);
    return bucket_of(x, thr, nthr);
  }
  return ld_i32(c, r);
}

template <typename T>
__device__ __forceinline__ void atomic_add_out(double *p, T v) { atomicAdd(p, (double)v); }

__device__ __forceinline__ int64_t seg_digit(const DSegment &s, int64_t seg, int i) {
  return (seg / s.radix[i]) % s.dom[i];
}

__device__ __forceinline__ int64_t outer_key(const DOuter &o, const DSegment &s, int64_t seg) {
  int64_t k = 0;
  for (int i = 0; i < s.ndig; ++i)
    if (o.dstride[i]) k += seg_digit(s, seg, i) * o.dstride[i];
  return k;
}

// ------------------------------------------------------------------ view kernel
// grid (tiles of rows, column groups): CTA (x, y) computes the y-th run of consecutive view
// columns for a tile of rows of r (one thread per row: coalesced reads of r's columns, uniform
// column descriptors, and a row's columns of a run written by one thread); the number of runs
// gives large relations one run (each row's key and child lookups done once) and small ones a
// run per column (enough threads); the last run also writes the group codes
__global__ void __launch_bounds__(256) view_kernel(DViewKernel d) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= d.nrows) return;
  int64_t k = 0;
  for (int i = 0; i < d.nk; ++i) k += (int64_t)ld_i32(d.in[d.kcol[i]], r) * d.kstride[i];
  int64_t ck[MAXCH];
  double w = 1.0;
  for (int c = 0; c < d.nchild; ++c) {
    const DViewRef &v = d.child[c];
    int64_t kk = 0;
    for (int i = 0; i < v.nk; ++i) kk += (int64_t)ld_i32(d.in[v.kcol[i]], r) * v.kstride[i];
    ck[c] = kk;
    w *= __ldg(v.v64 + kk * v.ncols);
  }
  if (w == 0.0) return;  // the tuple has no partner in some child: it does not join
  const int run = (d.ncols + gridDim.y - 1) / gridDim.y;
  const int j1 = min(d.ncols, (int)(blockIdx.y + 1) * run);
  for (int j = blockIdx.y * run; j < j1; ++j) {
    double val = 1.0;
    for (int f = d.col_fac_off[j]; f < d.col_fac_off[j + 1]; ++f) val *= fac_at<double>(d.in, d.facs[f], r);
    for (int p = d.col_part_off[j]; p < d.col_part_off[j + 1]; ++p) {
      const int2 pp = d.parts[p];
      val *= __ldg(d.child[pp.x].v64 + ck[pp.x] * d.child[pp.x].ncols + pp.y);
    }
    double *cell = d.v64 + k * d.ncols + j;
    if (d.unique) *cell = val;
    else if (val != 0.0) atomicAdd(cell, val);
  }
  if (blockIdx.y != gridDim.y - 1 || d.ncodes == 0) return;
  for (int c = 0; c < d.ncodes; ++c) {
    int4 cd = d.code_desc[c];
    int code;
    if (cd.x >= 0) {
      code = code_at(d.in[cd.x], r, cd.y, d.thr + cd.z, cd.w);
    } else {
      int2 ch = d.code_child[c];
      code = __ldg(d.child[ch.x].codes + ck[ch.x] * d.child[ch.x].ncodes + ch.y);
    }
    int old = atomicCAS(d.codes + k * d.ncodes + c, -1, code);
    if (old != -1 && old != code) atomicOr(d.err, 1);
  }
}

// Key-major form with one thread per key (kb consecutive keys per CTA): the column
// descriptors are staged in shared memory, the thread reads its row's input columns once and
// forms every view column of the key in a shared tile; the CTA then writes its keys' rows,
// which are one contiguous span of the view, with coalesced stores.
__global__ void __launch_bounds__(128) view_key_rows_kernel(DViewKernel d, int kb) {
  extern __shared__ __align__(16) unsigned char vsm[];
  const int tid = threadIdx.x;
  const int w = d.ncols + 1;
  double *vtile = reinterpret_cast<double *>(vsm);  // [kb][ncols + 1]
  int *scfo = reinterpret_cast<int *>(vtile + (size_t)kb * w);
  const int nfac = d.col_fac_off[d.ncols];
  DFac *sfac = reinterpret_cast<DFac *>(scfo + ((d.ncols + 1 + 3) & ~3));
  for (int i = tid; i <= d.ncols; i += blockDim.x) scfo[i] = d.col_fac_off[i];
  for (int i = tid; i < nfac; i += blockDim.x) sfac[i] = d.facs[i];
  __syncthreads();
  const int64_t k0 = (int64_t)blockIdx.x * kb;
  const int nk = (int)(d.nkeys - k0 < kb ? d.nkeys - k0 : kb);
  for (int t = tid; t < nk; t += blockDim.x) {
    const int64_t k = k0 + t;
    const int r = __ldg(d.keyrow + k);
    bool live = r >= 0;
    int64_t ck[MAXCH];
    double xin[MAXRC];
    if (live) {
      for (int c = 0; c < d.ncolsin; ++c) xin[c] = ld_num<double>(d.in[c], r);
      for (int c = 0; c < d.nchild; ++c) {
        const DViewRef &v = d.child[c];
        int64_t kk = 0;
        for (int i = 0; i < v.nk; ++i) kk += (int64_t)ld_i32(d.in[v.kcol[i]], r) * v.kstride[i];
        ck[c] = kk;
        if (__ldg(v.v64 + kk * v.ncols) == 0.0) live = false;  // no partner in this child
      }
    }
    for (int j = 0; j < d.ncols; ++j) {
      double val = 0.0;
      if (live) {
        val = 1.0;
        for (int f = scfo[j]; f < scfo[j + 1]; ++f) {
          const DFac fc = sfac[f];
          const double x = xin[fc.col];
          if (fc.ind) {
            // predicates compare the stored value: FP32 columns in FP32, integer columns exactly
            const bool ok = d.in[fc.col].dtype == LMFAO_F32 ? cmp_op<float>((float)x, fc.t, fc.op)
                                                            : cmp_op<double>(x, (double)fc.t, fc.op);
            val *= ok ? 1.0 : 0.0;
          } else {
            double v = x;
            for (int p = 1; p < fc.pow; ++p) v *= x;
            val *= v;
          }
        }
        for (int p = d.col_part_off[j]; p < d.col_part_off[j + 1]; ++p) {
          const int2 pp = d.parts[p];
          val *= __ldg(d.child[pp.x].v64 + ck[pp.x] * d.child[pp.x].ncols + pp.y);
        }
      }
      vtile[t * w + j] = val;
    }
    for (int c = 0; c < d.ncodes; ++c) {
      int code = -1;
      if (live) {
        const int4 cd = d.code_desc[c];
        if (cd.x >= 0) {
          code = code_at(d.in[cd.x], r, cd.y, d.thr + cd.z, cd.w);
        } else {
          const int2 ch = d.code_child[c];
          code = __ldg(d.child[ch.x].codes + ck[ch.x] * d.child[ch.x].ncodes + ch.y);
        }
      }
      d.codes[k * d.ncodes + c] = code;
    }
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  double *out = d.v64 + k0 * d.ncols;
  for (int t = warp; t < nk; t += nwarp)
    for (int j = lane; j < d.ncols; j += 32) out[(int64_t)t * d.ncols + j] = vtile[t * w + j];
}

__global__ void view_finish_kernel(const double *v64, float *v32, uint32_t *vint, const int *intcols,
                                   int ncols, int nint, int64_t nkeys, int *err) {
  const int64_t n = nkeys * ncols;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if (v32)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v32[i] = (float)v64[i];
  const int64_t ni = nkeys * nint;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += stride) {
    int64_t k = i / nint;
    int c = (int)(i % nint);
    double x = v64[k * ncols + intcols[c]];
    if (x >= 4294967296.0) atomicOr(err, 2);
    vint[i] = (uint32_t)x;
  }
}

// ------------------------------------------------------------------ segment weights
__global__ void segment_weight_kernel(DSegWeight d) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < d.nseg; s += stride) {
    unsigned long long w = 1;
    for (int o = 0; o < d.nouter; ++o) {
      int64_t k = outer_key(d.outer[o], d.seg, s);
      w *= (unsigned long long)__ldg(d.outer[o].v.v64 + k * d.outer[o].v.ncols);
    }
    d.wseg[s] = w;
  }
}

// ------------------------------------------------------------------ outer terms
// psi = segment-key factors x product of outer view columns (float and integral forms)
template <typename T>
__device__ __forceinline__ void eval_psi(const DPsi &p, const DSegFac *sf, const DPart *pp,
                                         const DOuter *outer, const DSegment &sg, int64_t seg,
                                         T &vf, unsigned long long &vi) {
  T v = T(1);
  unsigned long long iv = 1;
  for (int f = p.f0; f < p.f0 + p.nf; ++f) {
    DSegFac q = sf[f];
    int64_t dgt = seg_digit(sg, seg, q.digit);
    if (q.ind) {
      bool ok = cmp_op<double>((double)dgt, (double)q.t, q.op);
      if (!ok) { v = T(0); iv = 0; }
    } else {
      T x = (T)dgt, y = x;
      for (int e = 1; e < q.pow; ++e) y *= x;
      v *= y;
    }
  }
  for (int i = p.p0; i < p.p0 + p.np; ++i) {
    DPart q = pp[i];
    const DOuter &o = outer[q.branch];
    int64_t k = outer_key(o, sg, seg);
    double x = __ldg(o.v.v64 + k * o.v.ncols + q.col);
    if (p.integral) iv *= (unsigned long long)x;
    else v *= (T)x;
  }
  vf = v;
  vi = iv;
}

__device__ __forceinline__ int64_t outer_cell(const DGroupRef *g, int n, const DOuter *outer,
                                             const DSegment &sg, int64_t seg, bool &ok) {
  int64_t cell = 0;
  for (int i = 0; i < n; ++i) {
    DGroupRef q = g[i];
    int64_t code;
    if (q.src == 0) {
      code = seg_digit(sg, seg, q.a);
    } else {
      const DOuter &o = outer[q.a];
      int64_t k = outer_key(o, sg, seg);
      code = __ldg(o.v.codes + k * o.v.ncodes + q.b);
    }
    if (code < 0) ok = false;
    cell += code * q.stride;
  }
  return cell;
}

// ------------------------------------------------------------------ root fact pass
template <typename T>
__device__ __forceinline__ T rterm_f(const DFactPass &d, int t, const T *smf, const int *skx, int tid, int bs) {
  DRTerm rt = d.rt[t];
  T v = smf[rt.mono * bs + tid];
  for (int p = rt.p0; p < rt.p0 + rt.np; ++p) {
    DPart q = d.parts[p];
    const DViewRef &iv = d.inner[q.branch];
    int64_t k = skx[q.branch * bs + tid];
    if (sizeof(T) == 4) v *= (T)__ldg(iv.v32 + k * iv.ncols + q.col);
    else v *= (T)__ldg(iv.v64 + k * iv.ncols + q.col);
  }
  return v;
}

template <typename T>
__device__ __forceinline__ unsigned long long rterm_i(const DFactPass &d, int t, const unsigned char *smi,
                                                      const int *skx, int tid, int bs) {
  DRTerm rt = d.rt[t];
  unsigned long long v = smi[rt.mono * bs + tid];
  for (int p = rt.p0; p < rt.p0 + rt.np && v; ++p) {
    DPart q = d.parts[p];
    const DViewRef &iv = d.inner[q.branch];
    int64_t k = skx[q.branch * bs + tid];
    v *= (unsigned long long)__ldg(iv.vint + k * iv.nint + q.col);
  }
  return v;
}

template <typename T, int NB0>
__global__ void __launch_bounds__(256) fact_pass_kernel(DFactPass d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = bs >> 5;
  T *smf = reinterpret_cast<T *>(smem);                                 // nmono x bs
  int *skx = reinterpret_cast<int *>(smf + (size_t)d.nmono * bs);       // ninner x bs
  unsigned long long *wpsi_i =
      reinterpret_cast<unsigned long long *>(skx + (size_t)d.ninner * bs + ((d.ninner * bs) & 1));
  T *wpsi_f = reinterpret_cast<T *>(wpsi_i + (size_t)nwarps * d.b2_smem_items);
  long long *wocell = reinterpret_cast<long long *>(
      reinterpret_cast<unsigned char *>(wpsi_f) +
      (((size_t)nwarps * d.b2_smem_items * sizeof(T) + 7) & ~(size_t)7));
  unsigned char *smi = reinterpret_cast<unsigned char *>(wocell + (size_t)nwarps * d.b2_smem_items);

  for (int64_t w = (int64_t)blockIdx.x * nwarps + warp; w < d.nwork; w += (int64_t)gridDim.x * nwarps) {
    const DWork wk = d.work[w];
    const unsigned long long ws = d.wseg[wk.seg];
    if (ws == 0) continue;  // no outer partner: the whole segment drops out of the join
    // B2: outer terms and outer cells of this segment, staged per warp
    for (int i = lane; i < d.nb2; i += 32) {
      DB2Item it = d.b2[i];
      T pf;
      unsigned long long pi;
      eval_psi<T>(d.psi[it.psi], d.segfacs, d.psiparts, d.outer, d.seg, wk.seg, pf, pi);
      bool ok = true;
      long long oc = outer_cell(d.grefs + it.og0, it.nog, d.outer, d.seg, wk.seg, ok);
      wpsi_f[warp * d.b2_smem_items + i] = ok ? pf : T(0);
      wpsi_i[warp * d.b2_smem_items + i] = ok ? pi : 0ull;
      wocell[warp * d.b2_smem_items + i] = oc;
    }
    __syncwarp();
    T accf[NB0];
    unsigned long long acci[NI0_MAX];
#pragma unroll
    for (int j = 0; j < NB0; ++j) accf[j] = T(0);
#pragma unroll
    for (int j = 0; j < NI0_MAX; ++j) acci[j] = 0;
    const long long rend = wk.r0 + wk.len;
    for (long long r = wk.r0 + lane; r < rend; r += 32) {
      for (int b = 0; b < d.ninner; ++b) {
        const DViewRef &iv = d.inner[b];
        int64_t k = 0;
        for (int i = 0; i < iv.nk; ++i) k += (int64_t)ld_i32(d.col[iv.kcol[i]], r) * iv.kstride[i];
        skx[b * bs + tid] = (int)k;
      }
      for (int m = 0; m < d.nmono; ++m) {
        DMono mo = d.mono[m];
        T v = T(1);
        unsigned char ind = 1;
        for (int f = mo.f0; f < mo.f0 + mo.nf; ++f) {
          DFac fc = d.facs[f];
          T x = fac_at<T>(d.col, fc, r);
          v *= x;
          if (fc.ind && x == T(0)) ind = 0;
        }
        smf[m * bs + tid] = v;
        smi[m * bs + tid] = ind;
      }
#pragma unroll
      for (int j = 0; j < NB0; ++j)
        if (j < d.n0f) accf[j] += rterm_f<T>(d, d.b0f[j], smf, skx, tid, bs);
#pragma unroll
      for (int j = 0; j < NI0_MAX; ++j)
        if (j < d.n0i) acci[j] += rterm_i<T>(d, d.b0i[j], smi, skx, tid, bs);
      for (int i = 0; i < d.nb2; ++i) {
        DB2Item it = d.b2[i];
        double vf = 0.0;
        unsigned long long vi = 0;
        if (it.integral) {
          vi = wpsi_i[warp * d.b2_smem_items + i];
          if (vi) vi *= rterm_i<T>(d, it.rterm, smi, skx, tid, bs);
          if (!vi) continue;
        } else {
          T pf = wpsi_f[warp * d.b2_smem_items + i];
          if (pf == T(0)) continue;
          T v = pf * rterm_f<T>(d, it.rterm, smf, skx, tid, bs);
          if (v == T(0)) continue;
          vf = (double)v;
        }
        int64_t cell = wocell[warp * d.b2_smem_items + i];
        bool ok = true;
        for (int g = it.ig0; g < it.ig0 + it.nig; ++g) {
          DGroupRef q = d.grefs[g];
          int64_t code;
          if (q.src == 2) code = code_at(d.col[q.a], r, q.kind, d.thr + q.thr0, q.nthr);
          else code = __ldg(d.inner[q.a].codes + (int64_t)skx[q.a * bs + tid] * d.inner[q.a].ncodes + q.b);
          if (code < 0) ok = false;
          cell += code * q.stride;
        }
        if (!ok) continue;
        if (it.integral) atomicAdd(d.icnt + it.out + cell * it.cellmul, vi);
        else atomicAdd(d.fsum + it.out + cell * it.cellmul, vf);
      }
    }
    // per-segment sums: warp reduction, one atomic per column
#pragma unroll
    for (int j = 0; j < NB0; ++j) {
      if (j < d.n0f) {
        T v = accf[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v != T(0)) atomicAdd(reinterpret_cast<T *>(d.phi0f) + (int64_t)wk.seg * d.n0f + j, v);
      }
    }
#pragma unroll
    for (int j = 0; j < NI0_MAX; ++j) {
      if (j < d.n0i) {
        unsigned long long v = acci[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(d.phi0i + (int64_t)wk.seg * d.n0i + j, v);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ reorganisation
__global__ void segment_id_kernel(DCol c0, DCol c1, DCol c2, DCol c3, int ncols, int64_t r0, int64_t r1,
                                  int64_t r2, int64_t r3, int64_t n, int *segid) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    int64_t s = 0;
    if (ncols > 0) s += (int64_t)ld_i32(c0, r) * r0;
    if (ncols > 1) s += (int64_t)ld_i32(c1, r) * r1;
    if (ncols > 2) s += (int64_t)ld_i32(c2, r) * r2;
    if (ncols > 3) s += (int64_t)ld_i32(c3, r) * r3;
    segid[r] = (int)s;
  }
}

__global__ void histogram_kernel(const int *segid, int64_t n, unsigned int *hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
    atomicAdd(hist + segid[r], 1u);
}

struct DScatterCols {
  const void *in[MAXRC];
  void *out[MAXRC];
  int esz[MAXRC];
  int ncols;
};

__global__ void scatter_rows_kernel(const int *segid, int64_t n, unsigned long long *cursor, DScatterCols c,
                                    unsigned int *dest) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    unsigned long long pos = atomicAdd(cursor + segid[r], 1ull);
    if (dest) dest[r] = (unsigned int)pos;
    for (int j = 0; j < c.ncols; ++j) {
      if (c.esz[j] == 4) reinterpret_cast<int *>(c.out[j])[pos] = reinterpret_cast<const int *>(c.in[j])[r];
      else reinterpret_cast<unsigned char *>(c.out[j])[pos] = reinterpret_cast<const unsigned char *>(c.in[j])[r];
    }
  }
}

// out[dest[r]] = in[r]: a column moved into the segment order recorded by scatter_rows_kernel
__global__ void permute_rows_kernel(const unsigned int *dest, int64_t n, DScatterCols c) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const unsigned int pos = dest[r];
    for (int j = 0; j < c.ncols; ++j) {
      if (c.esz[j] == 4) reinterpret_cast<int *>(c.out[j])[pos] = reinterpret_cast<const int *>(c.in[j])[r];
      else reinterpret_cast<unsigned char *>(c.out[j])[pos] = reinterpret_cast<const unsigned char *>(c.in[j])[r];
    }
  }
}

__global__ void range_check_kernel(const int *p, int64_t n, int64_t domain, int *bad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    int v = p[r];
    if (v < 0 || (int64_t)v >= domain) atomicOr(bad, 1);
  }
}

// row of each key of a relation whose keys are unique (keyrow is -1 beforehand)
__global__ void key_row_kernel(DScatterCols cols, const int64_t *stride_k, int64_t n, int *keyrow) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    int64_t k = 0;
    for (int j = 0; j < cols.ncols; ++j) k += (int64_t)reinterpret_cast<const int *>(cols.in[j])[r] * stride_k[j];
    keyrow[k] = (int)r;
  }
}

__global__ void key_mult_kernel(DScatterCols cols, const int64_t *stride_k, int64_t n, unsigned int *hist) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    int64_t k = 0;
    for (int j = 0; j < cols.ncols; ++j) k += (int64_t)reinterpret_cast<const int *>(cols.in[j])[r] * stride_k[j];
    atomicAdd(hist + k, 1u);
  }
}

__global__ void max_u32_kernel(const unsigned int *h, int64_t n, unsigned int *out) {
  unsigned int m = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) m = max(m, h[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ------------------------------------------------------------------ results
__global__ void results_kernel(const unsigned long long *icnt, const double *fsum, int64_t cells, int naggs,
                               const int *integral, int64_t *counts, double *sums) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += stride) {
    if (counts) counts[c] = (int64_t)icnt[c * (1 + naggs)];
    if (sums)
      for (int a = 0; a < naggs; ++a)
        sums[c * naggs + a] = integral[a] ? (double)icnt[c * (1 + naggs) + 1 + a] : fsum[c * naggs + a];
  }
}

// CART: qdesc per query = (icnt base, fsum base, nbuckets, naggs, sum agg index, sumsq agg index,
// flags) -- the COUNT comes from icnt[cell*(1+naggs)], SUM(y) and SUM(y^2) from fsum.
__global__ void cart_kernel(const unsigned long long *icnt, const double *fsum, const int64_t *qdesc, int n,
                            int nb_max, double *out) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const int64_t *qd = qdesc + q * 6;
  int64_t ib = qd[0], fb = qd[1];
  int nb = (int)qd[2], na = (int)qd[3], a1 = (int)qd[4], a2 = (int)qd[5];
  double totn = 0, tots = 0, tots2 = 0;
  for (int b = 0; b < nb; ++b) {
    totn += (double)icnt[ib + (int64_t)b * (1 + na)];
    tots += fsum[fb + (int64_t)b * na + a1];
    tots2 += fsum[fb + (int64_t)b * na + a2];
  }
  double cn = 0, cs = 0, cs2 = 0;
  for (int b = 0; b + 1 < nb; ++b) {
    cn += (double)icnt[ib + (int64_t)b * (1 + na)];
    cs += fsum[fb + (int64_t)b * na + a1];
    cs2 += fsum[fb + (int64_t)b * na + a2];
    double rn = totn - cn, rs = tots - cs, rs2 = tots2 - cs2;
    out[((int64_t)q * (nb_max - 1) + b) * 2 + 0] = cn > 0 ? cs2 - cs * cs / cn : 0.0;
    out[((int64_t)q * (nb_max - 1) + b) * 2 + 1] = rn > 0 ? rs2 - rs * rs / rn : 0.0;
  }
}

// Best CART split per node (Section 3, decision trees): the queries of node v are
// qdesc[qbeg[v] .. qbeg[v+1]) (one per feature, in feature order), each a bucketed
// (COUNT, SUM(y), SUM(y^2)) query. A split "bucket <= k" of a query is valid when both
// sides hold tuples; its score is VARIANCE(left) + VARIANCE(right) in FP64. The least
// score wins, ties going to the earlier query, then the lower threshold. One CTA per node.
__global__ void __launch_bounds__(256) cart_split_kernel(const unsigned long long *icnt, const double *fsum,
                                                         const int64_t *qdesc, const int *qbeg, int2 *best,
                                                         double *score, double *stats) {
  const int v = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q0 = qbeg[v], q1 = qbeg[v + 1];
  double bs = 0.0;
  int bq = -1, bk = -1;
  // lanes over thresholds of one query per warp (at most 32 buckets per query here; more are
  // handled by striding k)
  for (int q = q0 + warp; q < q1; q += blockDim.x >> 5) {
    const int64_t *qd = qdesc + (int64_t)q * 6;
    const int64_t ib = qd[0], fb = qd[1];
    const int nb = (int)qd[2], na = (int)qd[3], a1 = (int)qd[4], a2 = (int)qd[5];
    double tn = 0, ts = 0, ts2 = 0;
    for (int b = 0; b < nb; ++b) {
      tn += (double)icnt[ib + (int64_t)b * (1 + na)];
      ts += fsum[fb + (int64_t)b * na + a1];
      ts2 += fsum[fb + (int64_t)b * na + a2];
    }
    if (q == q0 && lane == 0 && stats) {
      stats[3 * v + 0] = tn;
      stats[3 * v + 1] = ts;
      stats[3 * v + 2] = ts2;
    }
    for (int k = lane; k + 1 < nb; k += 32) {
      double cn = 0, cs = 0, cs2 = 0;
      for (int b = 0; b <= k; ++b) {
        cn += (double)icnt[ib + (int64_t)b * (1 + na)];
        cs += fsum[fb + (int64_t)b * na + a1];
        cs2 += fsum[fb + (int64_t)b * na + a2];
      }
      const double rn = tn - cn;
      if (cn <= 0 || rn <= 0) continue;
      const double sc = (cs2 - cs * cs / cn) + ((ts2 - cs2) - (ts - cs) * (ts - cs) / rn);
      if (bq < 0 || sc < bs || (sc == bs && (q < bq || (q == bq && k < bk)))) { bs = sc; bq = q; bk = k; }
    }
  }
  // CTA argmin with the same order
  __shared__ double ss[256];
  __shared__ int sq[256], sk[256];
  ss[tid] = bs;
  sq[tid] = bq;
  sk[tid] = bk;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) {
      const double os = ss[tid + w];
      const int oq = sq[tid + w], ok = sk[tid + w];
      const bool take = oq >= 0 && (sq[tid] < 0 || os < ss[tid] ||
                                    (os == ss[tid] && (oq < sq[tid] || (oq == sq[tid] && ok < sk[tid]))));
      if (take) { ss[tid] = os; sq[tid] = oq; sk[tid] = ok; }
    }
    __syncthreads();
  }
  if (tid == 0) {
    best[v] = make_int2(sq[0] < 0 ? -1 : sq[0] - q0, sk[0]);
    score[v] = sq[0] < 0 ? 0.0 : ss[0];
  }
}

// Ridge regression from the aggregates of one query (Section 3, linear regression): z = (1,
// x_1 .. x_d, y); zmap[i * (d + 2) + j] is the aggregate of SUM(z_i z_j) (-1: the COUNT).
// A = SUM(x x^T) / n + lambda I, b = SUM(x y) / n (x = z_0 .. z_d); the closed form solves
// A theta = b by Cholesky; batch gradient descent takes `iters` steps theta -= step * (A theta - b)
// from theta = 0. out: theta (d + 1), then J(theta), then |A theta - b|. One CTA, FP64.
__global__ void __launch_bounds__(256) ridge_kernel(const unsigned long long *icnt, const double *fsum,
                                                    int64_t io, int64_t fo, const int *zmap, int d, double lambda,
                                                    int method, int iters, double step, double *out) {
  extern __shared__ double rs[];
  const int m = d + 1, w = d + 2, tid = threadIdx.x, bs = blockDim.x;
  double *A = rs;            // m x m
  double *L = A + m * m;     // m x m (Cholesky factor)
  double *b = L + m * m;     // m
  double *th = b + m;        // m
  double *g = th + m;        // m
  double *syy = g + m;       // 1
  const double n = (double)icnt[io];
  for (int idx = tid; idx < w * w; idx += bs) {
    const int i = idx / w, j = idx - i * w;
    const int a = zmap[idx];
    const double v = a < 0 ? n : fsum[fo + a];
    if (i < m && j < m) A[i * m + j] = v / n + (i == j ? lambda : 0.0);
    else if (i < m && j == m) b[i] = v / n;
    else if (i == m && j == m) syy[0] = v / n;
  }
  for (int i = tid; i < m; i += bs) th[i] = 0.0;
  __syncthreads();
  if (method == 0) {
    // Cholesky A = L L^T, column by column
    for (int i = tid; i < m * m; i += bs) L[i] = 0.0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
      if (tid == 0) {
        double s = A[k * m + k];
        for (int p = 0; p < k; ++p) s -= L[k * m + p] * L[k * m + p];
        L[k * m + k] = sqrt(s > 0 ? s : 0.0);
      }
      __syncthreads();
      for (int i = k + 1 + tid; i < m; i += bs) {
        double s = A[i * m + k];
        for (int p = 0; p < k; ++p) s -= L[i * m + p] * L[k * m + p];
        L[i * m + k] = L[k * m + k] > 0 ? s / L[k * m + k] : 0.0;
      }
      __syncthreads();
    }
    if (tid == 0) {  // L u = b, then L^T theta = u
      for (int i = 0; i < m; ++i) {
        double s = b[i];
        for (int p = 0; p < i; ++p) s -= L[i * m + p] * g[p];
        g[i] = L[i * m + i] > 0 ? s / L[i * m + i] : 0.0;
      }
      for (int i = m - 1; i >= 0; --i) {
        double s = g[i];
        for (int p = i + 1; p < m; ++p) s -= L[p * m + i] * th[p];
        th[i] = L[i * m + i] > 0 ? s / L[i * m + i] : 0.0;
      }
    }
    __syncthreads();
  } else {
    for (int it = 0; it < iters; ++it) {
      for (int i = tid; i < m; i += bs) {
        double s = -b[i];
        for (int j = 0; j < m; ++j) s += A[i * m + j] * th[j];
        g[i] = s;
      }
      __syncthreads();
      for (int i = tid; i < m; i += bs) th[i] -= step * g[i];
      __syncthreads();
    }
  }
  // gradient and objective at theta: J = (theta^T (A - lambda I) theta - 2 theta^T b + syy) / 2
  //                                      + lambda / 2 |theta|^2 = (theta^T A theta - 2 theta^T b + syy) / 2
  for (int i = tid; i < m; i += bs) {
    double s = -b[i];
    for (int j = 0; j < m; ++j) s += A[i * m + j] * th[j];
    g[i] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double q = 0, tb = 0, gn = 0;
    for (int i = 0; i < m; ++i) {
      q += th[i] * (g[i] + b[i]);
      tb += th[i] * b[i];
      gn += g[i] * g[i];
    }
    for (int i = 0; i < m; ++i) out[i] = th[i];
    out[m] = 0.5 * (q - 2.0 * tb + syy[0]);
    out[m + 1] = sqrt(gn);
  }
}

// ------------------------------------------------------------------ launchers
static int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  if (g > 148 * 32) g = 148 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

size_t view_key_rows_smem(const DViewKernel &d) {
  return (size_t)kVkb * (d.ncols + 1) * 8 + 4 * (size_t)((d.ncols + 1 + 3) & ~3) + sizeof(DFac) * (size_t)d.nfac;
}

void launch_view_kernel(const DViewKernel &d, cudaStream_t s) {
  if (d.keyrow) {  // the plan gives a key-row map only to views whose key tile fits (view_key_rows_smem)
    const size_t sm = view_key_rows_smem(d);
    if (d.nkeys) view_key_rows_kernel<<<(unsigned)((d.nkeys + kVkb - 1) / kVkb), kVkb, sm, s>>>(d, kVkb);
    return;
  }
  if (d.nrows == 0) return;
  // enough rows x runs to fill 148 SMs x 2048 threads, and no more runs than that
  const int64_t want = (148LL * 2048 + d.nrows - 1) / d.nrows;
  const int groups = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(d.ncols, 65535), want));
  view_kernel<<<dim3((unsigned)((d.nrows + 255) / 256), groups), 256, 0, s>>>(d);
}

void launch_view_finish(const double *v64, float *v32, uint32_t *vint, const int *intcols, int ncols, int nint,
                        int64_t nkeys, int *err, cudaStream_t s) {
  const int64_t n = std::max<int64_t>(v32 ? nkeys * (int64_t)ncols : 0, nkeys * (int64_t)nint);
  if (n == 0) return;
  view_finish_kernel<<<grid_for(n, 256), 256, 0, s>>>(v64, v32, vint, intcols, ncols, nint, nkeys, err);
}

void launch_segment_weights(const DSegWeight &d, cudaStream_t s) {
  segment_weight_kernel<<<grid_for(d.nseg, 256), 256, 0, s>>>(d);
}

template <typename T>
static void launch_fp(const DFactPass &d, int nb0, int grid, int block, size_t smem, cudaStream_t s) {
#define LMFAO_FP_CASE(N)                                                                              \
  case N:                                                                                             \
    cudaFuncSetAttribute(fact_pass_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    fact_pass_kernel<T, N><<<grid, block, smem, s>>>(d);                                              \
    break;
  switch (nb0) {
    LMFAO_FP_CASE(4)
    LMFAO_FP_CASE(8)
    LMFAO_FP_CASE(16)
    LMFAO_FP_CASE(32)
    LMFAO_FP_CASE(64)
    default: break;
  }
#undef LMFAO_FP_CASE
}

size_t fact_pass_smem(const DFactPass &d, bool fp64, int block) {
  size_t ts = fp64 ? 8 : 4;
  size_t nw = block / 32;
  size_t b = (size_t)d.nmono * block * ts;
  b += (size_t)d.ninner * block * 4 + (((size_t)d.ninner * block) & 1) * 4;
  b += nw * d.b2_smem_items * 8;
  b += (nw * d.b2_smem_items * ts + 7) & ~(size_t)7;
  b += nw * d.b2_smem_items * 8;
  b += (size_t)d.nmono * block;
  return b;
}

void launch_fact_pass(const DFactPass &d, bool fp64, int nb0, int grid, int block, cudaStream_t s) {
  size_t smem = fact_pass_smem(d, fp64, block);
  if (fp64) launch_fp<double>(d, nb0, grid, block, smem, s);
  else launch_fp<float>(d, nb0, grid, block, smem, s);
}

void launch_segment_ids(const DCol *cols, int ncols, const int64_t *radix, int64_t n, int *segid, cudaStream_t s) {
  DCol c[4] = {};
  int64_t r[4] = {0, 0, 0, 0};
  for (int i = 0; i < ncols && i < 4; ++i) { c[i] = cols[i]; r[i] = radix[i]; }
  segment_id_kernel<<<grid_for(n, 256), 256, 0, s>>>(c[0], c[1], c[2], c[3], ncols, r[0], r[1], r[2], r[3], n, segid);
}

void launch_histogram(const int *segid, int64_t n, unsigned int *hist, cudaStream_t s) {
  histogram_kernel<<<grid_for(n, 256), 256, 0, s>>>(segid, n, hist);
}

void launch_scatter_rows(const int *segid, int64_t n, unsigned long long *cursor, const DCol *in, DCol *out,
                         const int *elem_size, int ncols, unsigned int *dest, cudaStream_t s) {
  DScatterCols c{};
  c.ncols = ncols;
  for (int j = 0; j < ncols; ++j) { c.in[j] = in[j].p; c.out[j] = const_cast<void *>(out[j].p); c.esz[j] = elem_size[j]; }
  scatter_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(segid, n, cursor, c, dest);
}

void launch_permute_rows(const unsigned int *dest, int64_t n, const DCol *in, DCol *out, const int *elem_size,
                         int ncols, cudaStream_t s) {
  if (n == 0 || ncols == 0) return;
  DScatterCols c{};
  c.ncols = ncols;
  for (int j = 0; j < ncols; ++j) { c.in[j] = in[j].p; c.out[j] = const_cast<void *>(out[j].p); c.esz[j] = elem_size[j]; }
  permute_rows_kernel<<<grid_for(n, 256), 256, 0, s>>>(dest, n, c);
}

void launch_range_check(const void *p, int dtype, int64_t n, int64_t domain, int *bad, cudaStream_t s) {
  (void)dtype;
  if (n == 0) return;
  range_check_kernel<<<grid_for(n, 256), 256, 0, s>>>(reinterpret_cast<const int *>(p), n, domain, bad);
}

void launch_key_multiplicity(const DCol *cols, int ncols, const int64_t *stride, int64_t n, unsigned int *hist,
                             cudaStream_t s) {
  if (n == 0) return;
  DScatterCols c{};
  c.ncols = ncols;
  for (int j = 0; j < ncols; ++j) c.in[j] = cols[j].p;
  key_mult_kernel<<<grid_for(n, 256), 256, 0, s>>>(c, stride, n, hist);
}

void launch_key_rows(const DCol *cols, int ncols, const int64_t *stride, int64_t n, int *keyrow, cudaStream_t s) {
  if (n == 0) return;
  DScatterCols c{};
  c.ncols = ncols;
  for (int j = 0; j < ncols; ++j) c.in[j] = cols[j].p;
  key_row_kernel<<<grid_for(n, 256), 256, 0, s>>>(c, stride, n, keyrow);
}

void launch_max_u32(const unsigned int *h, int64_t n, unsigned int *out, cudaStream_t s) {
  if (n == 0) return;
  max_u32_kernel<<<grid_for(n, 256), 256, 0, s>>>(h, n, out);
}

void launch_cart_variances(const unsigned long long *icnt, const double *fsum, const int64_t *qdesc, int n,
                           int nb_max, double *out, cudaStream_t s) {
  if (n == 0) return;
  cart_kernel<<<(n + 127) / 128, 128, 0, s>>>(icnt, fsum, qdesc, n, nb_max, out);
}

void launch_cart_split(const unsigned long long *icnt, const double *fsum, const int64_t *qdesc, const int *qbeg,
                       int nnodes, int2 *best, double *score, double *stats, cudaStream_t s) {
  if (nnodes == 0) return;
  cart_split_kernel<<<nnodes, 256, 0, s>>>(icnt, fsum, qdesc, qbeg, best, score, stats);
}

void launch_ridge(const unsigned long long *icnt, const double *fsum, int64_t io, int64_t fo, const int *zmap, int d,
                  double lambda, int method, int iters, double step, double *out, cudaStream_t s) {
  const int m = d + 1;
  const size_t smem = (size_t)(2 * m * m + 3 * m + 1) * sizeof(double);
  cudaFuncSetAttribute(ridge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  ridge_kernel<<<1, 256, smem, s>>>(icnt, fsum, io, fo, zmap, d, lambda, method, iters, step, out);
}

void launch_results(const unsigned long long *icnt, const double *fsum, int64_t cells, int naggs, const int *integral,
                    int64_t *counts, double *sums, cudaStream_t s) {
  if (cells == 0) return;
  results_kernel<<<grid_for(cells, 256), 256, 0, s>>>(icnt, fsum, cells, naggs, integral, counts, sums);
}

}  // namespace lmfao
