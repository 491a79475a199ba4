// Root pass for plans with at most one inner child (see fastpass.cuh) and the B3
// finalisation over the inner relation's keys.
#include <cuda_runtime.h>

#include "fastpass.cuh"

namespace lmfao {

namespace {

__device__ __forceinline__ int ldi(const DCol &c, int64_t r) { return __ldg(reinterpret_cast<const int *>(c.p) + r); }

template <typename T>
__device__ __forceinline__ T ldn(const DCol &c, int64_t r) {
  if (c.dtype == LMFAO_F32) return (T)__ldg(reinterpret_cast<const float *>(c.p) + r);
  if (c.dtype == LMFAO_U8) return (T)__ldg(reinterpret_cast<const unsigned char *>(c.p) + r);
  return (T)__ldg(reinterpret_cast<const int *>(c.p) + r);
}

template <typename X>
__device__ __forceinline__ bool cmpx(X x, X t, int op) {
  switch (op) {
    case LMFAO_LE: return x <= t;
    case LMFAO_LT: return x < t;
    case LMFAO_GE: return x >= t;
    case LMFAO_GT: return x > t;
    case LMFAO_EQ: return x == t;
    default: return x != t;
  }
}

// predicate on the stored value (FP32 compare for float columns, exact for integers)
__device__ __forceinline__ bool pred(const DCol &c, int64_t r, int op, float t) {
  if (c.dtype == LMFAO_F32) return cmpx<float>(__ldg(reinterpret_cast<const float *>(c.p) + r), t, op);
  double x = (c.dtype == LMFAO_U8) ? (double)__ldg(reinterpret_cast<const unsigned char *>(c.p) + r)
                                   : (double)__ldg(reinterpret_cast<const int *>(c.p) + r);
  return cmpx<double>(x, (double)t, op);
}

__device__ __forceinline__ int bucket(float x, const float *thr, int n) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(thr + mid) < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int row_code(const DCol &c, int64_t r, int kind, const float *thr, int nthr) {
  if (kind == LMFAO_GB_BUCKET) {
    float x = (c.dtype == LMFAO_F32) ? __ldg(reinterpret_cast<const float *>(c.p) + r)
              : (c.dtype == LMFAO_U8) ? (float)__ldg(reinterpret_cast<const unsigned char *>(c.p) + r)
                                      : (float)__ldg(reinterpret_cast<const int *>(c.p) + r);
    return bucket(x, thr, nthr);
  }
  return ldi(c, r);
}

template <int N, typename T>
__device__ __forceinline__ T sel(const T (&a)[N], int i) {
  T r = T(0);
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (k == i) r = a[k];
  return r;
}

template <typename T>
__global__ void fast_prep_kernel(int64_t nkeys, const double *v64, int vcols, const int *wcol, int nw, T *table,
                                 const int32_t *vcodes, int vncodes, const int *codecol, int ncode, int *codes) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nkeys; k += stride) {
    for (int w = 0; w < nw; ++w) table[k * nw + w] = (T)v64[k * vcols + wcol[w]];
    for (int c = 0; c < ncode; ++c) codes[k * ncode + c] = vcodes[k * vncodes + codecol[c]];
  }
}

template <typename T, int NM, int W>
__global__ void __launch_bounds__(512) fast_pass_kernel(DFast d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = bs >> 5;
  // shared layout: [Pf T nkeys*n3][Pi u32 nkeys*n3][table T nkeys*nw][codes int nkeys*ncode][warp hists]
  size_t off = 0;
  T *Pf = reinterpret_cast<T *>(smem);
  unsigned int *Pi = nullptr;
  if (d.smem_p) {
    off += sizeof(T) * (size_t)d.nkeys * d.n3;
    Pi = reinterpret_cast<unsigned int *>(smem + off);
    off += 4 * (size_t)d.nkeys * d.n3;
  }
  off = (off + 15) & ~(size_t)15;
  const T *table = reinterpret_cast<const T *>(d.table);
  const int *codes = d.codes;
  if (d.smem_view && d.ni) {
    T *st = reinterpret_cast<T *>(smem + off);
    off += sizeof(T) * (size_t)d.nkeys * d.nw;
    int *sc = reinterpret_cast<int *>(smem + off);
    off += 4 * (size_t)d.nkeys * d.ncode;
    for (int64_t i = tid; i < d.nkeys * d.nw; i += bs) st[i] = reinterpret_cast<const T *>(d.table)[i];
    for (int64_t i = tid; i < d.nkeys * d.ncode; i += bs) sc[i] = d.codes[i];
    table = st;
    codes = sc;
  }
  off = (off + 15) & ~(size_t)15;
  float *hf = reinterpret_cast<float *>(smem + off) + (size_t)warp * (d.hist_f + d.hist_i);
  unsigned int *hi = reinterpret_cast<unsigned int *>(hf + d.hist_f);
  if (d.smem_p)
    for (int64_t i = tid; i < d.nkeys * d.n3; i += bs) { Pf[i] = T(0); Pi[i] = 0u; }
  __syncthreads();

  for (int64_t wi = (int64_t)blockIdx.x * nwarps + warp; wi < d.nwork; wi += (int64_t)gridDim.x * nwarps) {
    const DWork wk = d.work[wi];
    const unsigned long long ws = d.wseg[wk.seg];
    if (ws == 0) continue;  // the whole segment has no outer partner
    const T wsT = (T)ws;
    if (d.nb1) {
      for (int i = lane; i < d.hist_f; i += 32) hf[i] = 0.f;
      for (int i = lane; i < d.hist_i; i += 32) hi[i] = 0u;
      __syncwarp();
    }
    T acc[NM][W];
#pragma unroll
    for (int j = 0; j < NM; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[j][w] = T(0);
    const long long rend = wk.r0 + wk.len;
    for (long long r = wk.r0 + lane; r < rend; r += 32) {
      int64_t k = 0;
      T v[W];
      if (d.ni) {
        for (int i = 0; i < d.nk; ++i) k += (int64_t)ldi(d.col[d.kslot[i]], r) * d.kstride[i];
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = (w < d.nw) ? table[k * d.nw + w] : T(0);
      } else {
        v[0] = T(1);
#pragma unroll
        for (int w = 1; w < W; ++w) v[w] = T(0);
      }
      if (v[0] == T(0)) continue;  // no partner in the inner relation: not in the join
      T x[FMAXX];
#pragma unroll
      for (int i = 0; i < FMAXX; ++i) x[i] = (i < d.nx) ? ldn<T>(d.col[d.xslot[i]], r) : T(0);
      T m[NM];
#pragma unroll
      for (int j = 0; j < NM; ++j) {
        T p = T(1);
        if (j < d.nm) {
          for (int f = d.mono_f0[j]; f < d.mono_f0[j] + d.mono_nf[j]; ++f) {
            const DFac fc = d.facs[f];
            if (fc.ind) {
              if (!pred(d.col[fc.col], r, fc.op, fc.t)) p = T(0);
            } else {
              T xv = sel<FMAXX, T>(x, d.fx[f]);
              T y = xv;
              for (int e = 1; e < fc.pow; ++e) y *= xv;
              p *= y;
            }
          }
        }
        m[j] = p;
      }
#pragma unroll
      for (int j = 0; j < NM; ++j)
#pragma unroll
        for (int w = 0; w < W; ++w) acc[j][w] += m[j] * v[w];
      for (int s = 0; s < d.nb1; ++s) {
        const DFastB1 &b = d.b1[s];
        int g = 0;
        bool ok = true;
        for (int i = 0; i < b.nref; ++i) {
          const DGroupRef &q = b.ref[i];
          int code = (q.src == 3) ? codes[k * d.ncode + q.b] : row_code(d.col[q.a], r, q.kind, d.thr + q.thr0, q.nthr);
          if (code < 0) ok = false;
          g += code * (int)q.stride;
        }
        if (!ok) continue;
        for (int c = 0; c < b.nf; ++c) {
          T val = sel<NM, T>(m, b.fj[c]) * sel<W, T>(v, b.fw[c]);
          if (val != T(0)) atomicAdd(hf + b.smem_f + g * b.nf + c, (float)val);
        }
        for (int c = 0; c < b.ni; ++c) {
          T val = sel<NM, T>(m, b.ij[c]) * sel<W, T>(v, b.iw[c]);
          if (val != T(0)) atomicAdd(hi + b.smem_i + g * b.ni + c, (unsigned int)val);
        }
      }
      for (int c = 0; c < d.n3; ++c) {
        T val = sel<NM, T>(m, d.j3[c]);
        if (val == T(0)) continue;
        if (d.int3[c]) {
          unsigned long long iv = (unsigned long long)val * ws;
          if (d.smem_p) atomicAdd(Pi + k * d.n3 + c, (unsigned int)iv);
          else atomicAdd(d.p3i + k * d.n3 + c, iv);
        } else {
          val *= wsT;
          if (d.smem_p) atomicAdd(Pf + k * d.n3 + c, val);
          else atomicAdd(d.p3f + k * d.n3 + c, (double)val);
        }
      }
    }
    // segment sums: warp reduction, then one atomic per entry
    const int n0 = d.nm * d.nw;
#pragma unroll
    for (int j = 0; j < NM; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) {
        if (j < d.nm && w < d.nw) {
          T t = acc[j][w];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          acc[j][w] = t;
          if (lane == ((j * W + w) & 31) && t != T(0))
            atomicAdd(reinterpret_cast<T *>(d.phi0f) + (int64_t)wk.seg * n0 + j * d.nw + w, t);
        }
      }
    if (lane < d.n0i) {
      T t = T(0);
#pragma unroll
      for (int j = 0; j < NM; ++j)
#pragma unroll
        for (int w = 0; w < W; ++w)
          if (j == d.i0j[lane] && w == d.i0w[lane]) t = acc[j][w];
      unsigned long long it = (unsigned long long)(t + T(0.5));
      if (it) atomicAdd(d.phi0i + (int64_t)wk.seg * d.n0i + lane, it);
    }
    if (d.nb1) {
      __syncwarp();
      for (int s = 0; s < d.nb1; ++s) {
        const DFastB1 &b = d.b1[s];
        for (int i = lane; i < b.G * b.nf; i += 32) {
          float x = hf[b.smem_f + i];
          if (x != 0.f) atomicAdd(d.phi1f + (int64_t)wk.seg * d.phi1f_seg + b.gbase_f + i, x);
        }
        for (int i = lane; i < b.G * b.ni; i += 32) {
          unsigned int x = hi[b.smem_i + i];
          if (x) atomicAdd(d.phi1i + (int64_t)wk.seg * d.phi1i_seg + b.gbase_i + i, x);
        }
      }
      __syncwarp();
    }
  }
  if (d.smem_p) {
    __syncthreads();
    for (int64_t i = tid; i < d.nkeys * d.n3; i += bs) {
      if (Pf[i] != T(0)) atomicAdd(d.p3f + i, (double)Pf[i]);
      if (Pi[i]) atomicAdd(d.p3i + i, (unsigned long long)Pi[i]);
    }
  }
}

__global__ void b3_final_kernel(DB3Final d) {
  const int64_t n = d.nkeys * d.nitems;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    int64_t k = idx / d.nitems;
    int it = (int)(idx - k * d.nitems);
    const DB3Item item = d.items[it];
    int64_t cell = 0;
    bool ok = true;
    for (int g = item.ig0; g < item.ig0 + item.nig; ++g) {
      DGroupRef q = d.grefs[g];
      int code = d.vcodes[k * d.vncodes + q.b];
      if (code < 0) ok = false;
      cell += (int64_t)code * q.stride;
    }
    if (!ok) continue;
    double vv = d.v64[k * d.vcols + item.w];
    if (vv == 0.0) continue;
    if (item.integral) {
      unsigned long long p = d.p3i[k * d.n3 + item.c];
      if (p) atomicAdd(d.icnt + item.out + cell * item.cellmul, p * (unsigned long long)vv);
    } else {
      double p = d.p3f[k * d.n3 + item.c];
      if (p != 0.0) atomicAdd(d.fsum + item.out + cell * item.cellmul, p * vv);
    }
  }
}

}  // namespace

void launch_fast_prep(const DFast &d, const double *v64, int vcols, const int *wcol, const int32_t *vcodes,
                      int vncodes, const int *codecol, void *table, int *codes, bool fp64, cudaStream_t s) {
  if (!d.ni || d.nkeys == 0) return;
  int grid = (int)std::min<int64_t>((d.nkeys + 255) / 256, 148 * 8);
  if (fp64)
    fast_prep_kernel<double><<<grid, 256, 0, s>>>(d.nkeys, v64, vcols, wcol, d.nw, (double *)table, vcodes, vncodes,
                                                   codecol, d.ncode, codes);
  else
    fast_prep_kernel<float><<<grid, 256, 0, s>>>(d.nkeys, v64, vcols, wcol, d.nw, (float *)table, vcodes, vncodes,
                                                  codecol, d.ncode, codes);
}

size_t fast_smem(const DFast &d, bool fp64, int block) {
  size_t ts = fp64 ? 8 : 4;
  size_t off = 0;
  if (d.smem_p) off += (ts + 4) * (size_t)d.nkeys * d.n3;
  off = (off + 15) & ~(size_t)15;
  if (d.smem_view && d.ni) off += ts * (size_t)d.nkeys * d.nw + 4 * (size_t)d.nkeys * d.ncode;
  off = (off + 15) & ~(size_t)15;
  off += (size_t)(block / 32) * (d.hist_f + d.hist_i) * 4;
  return off;
}

template <typename T, int NM, int W>
static void go(const DFast &d, int grid, int block, size_t smem, cudaStream_t s) {
  cudaFuncSetAttribute(fast_pass_kernel<T, NM, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  fast_pass_kernel<T, NM, W><<<grid, block, smem, s>>>(d);
}

template <typename T>
static bool dispatch(const DFast &d, int grid, int block, size_t smem, cudaStream_t s) {
  const int nm = d.nm, nw = d.nw;
#define LMFAO_FAST(M, Wd) \
  if (nm <= M && nw <= Wd) { go<T, M, Wd>(d, grid, block, smem, s); return true; }
  LMFAO_FAST(4, 1)
  LMFAO_FAST(8, 1)
  LMFAO_FAST(4, 2)
  LMFAO_FAST(4, 4)
  LMFAO_FAST(4, 8)
  LMFAO_FAST(8, 4)
  LMFAO_FAST(12, 4)
  LMFAO_FAST(16, 2)
  LMFAO_FAST(8, 8)
#undef LMFAO_FAST
  return false;
}

bool fast_shape_ok(int nm, int nw) {
  const int shapes[][2] = {{4, 1}, {8, 1}, {4, 2}, {4, 4}, {4, 8}, {8, 4}, {12, 4}, {16, 2}, {8, 8}};
  for (auto &sh : shapes)
    if (nm <= sh[0] && nw <= sh[1]) return true;
  return false;
}

bool launch_fast_pass(const DFast &d, bool fp64, int grid, int block, cudaStream_t s) {
  size_t smem = fast_smem(d, fp64, block);
  if (fp64) return dispatch<double>(d, grid, block, smem, s);
  return dispatch<float>(d, grid, block, smem, s);
}

void launch_b3_final(const DB3Final &d, cudaStream_t s) {
  int64_t n = d.nkeys * d.nitems;
  if (n == 0) return;
  int grid = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
  b3_final_kernel<<<grid, 256, 0, s>>>(d);
}

}  // namespace lmfao
