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
                                 const int32_t *vcodes, int vncodes, const int *codecol, int ncode, int *codes,
                                 const int2 *ib, int nib, int ibcode) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nkeys; k += stride) {
    for (int w = 0; w < nw; ++w) table[k * nw + w] = (T)v64[k * vcols + wcol[w]];
    for (int c = 0; c < ncode; ++c)
      if (c != ibcode) codes[k * ncode + c] = vcodes[k * vncodes + codecol[c]];
    if (ibcode >= 0) {  // inner predicate bits: the (unique) tuple of key k satisfies predicate j
      unsigned int bits = 0;
      for (int j = 0; j < nib; ++j)
        if (v64[k * vcols + ib[j].x] > 0.0) bits |= 1u << ib[j].y;
      codes[k * ncode + ibcode] = (int)bits;
    }
  }
}

template <typename T>
__device__ __forceinline__ T powu(T x, int e) {  // e is uniform across the warp
  T y = T(1);
  for (int k = 0; k < e; ++k) y *= x;
  return y;
}

constexpr int RU = 2;  // tuples per lane per step (their loads are issued first)

// Small descriptors of the per-tuple scatter work, copied to shared memory once per CTA.
struct SDesc {
  DFastB1 b1[FMAXB1];
  int j3[FMAXC], int3[FMAXC], p3col[FMAXC];
  DFac ind[FMAXF];
  int ind_mono[FMAXF];
};

template <typename T, int NM, int W>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512, 1) fast_pass_kernel(DFast d) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SDesc sd;
  const int bs = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = bs >> 5;
  // shared layout: [Pf T nkeys*n3][Pi u32 nkeys*n3][table T nkeys*nw][codes int nkeys*ncode][warp hists]
  size_t off = 0;
  T *Pf = reinterpret_cast<T *>(smem);
  unsigned int *Pi = nullptr;
  if (d.smem_p) {
    off += sizeof(T) * (size_t)d.nkeys * d.n3f * d.b3leaf;
    Pi = reinterpret_cast<unsigned int *>(smem + off);
    off += 4 * (size_t)d.nkeys * d.n3i * d.b3leaf;
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
  off += (size_t)nwarps * (d.hist_f + d.hist_i) * 4;
  off = (off + 15) & ~(size_t)15;
  T *b4f = reinterpret_cast<T *>(smem + off);  // CTA-private outputs of B4 items
  off += sizeof(T) * (size_t)d.b4_fcells;
  off = (off + 15) & ~(size_t)15;
  unsigned int *b4i = reinterpret_cast<unsigned int *>(smem + off);
  for (int i = tid; i < d.b4_fcells; i += bs) b4f[i] = T(0);
  for (int i = tid; i < d.b4_icells; i += bs) b4i[i] = 0u;
  if (d.smem_p) {
    for (int64_t i = tid; i < d.nkeys * d.n3f * d.b3leaf; i += bs) Pf[i] = T(0);
    for (int64_t i = tid; i < d.nkeys * d.n3i * d.b3leaf; i += bs) Pi[i] = 0u;
  }
  if (tid == 0) {
    for (int s = 0; s < FMAXB1; ++s) sd.b1[s] = d.b1[s];
    for (int c = 0; c < FMAXC; ++c) { sd.j3[c] = d.j3[c]; sd.int3[c] = d.int3[c]; sd.p3col[c] = d.p3col[c]; }
    for (int f = 0; f < FMAXF; ++f) { sd.ind[f] = d.ind[f]; sd.ind_mono[f] = d.ind_mono[f]; }
  }
  __syncthreads();
  const int nb1 = d.nb1, n3 = d.n3, nind = d.nind, nx = d.nx, nw = d.nw, ncode = d.ncode;
  const int n3f = d.n3f, n3i = d.n3i;

  for (;;) {
    int64_t wi = 0;
    if (lane == 0) wi = atomicAdd(d.ticket, 1u);
    wi = __shfl_sync(0xffffffffu, wi, 0);
    if (wi >= d.nwork) break;
    const DWork wk = d.work[wi];
    const unsigned long long ws = d.wseg[wk.seg];
    if (ws == 0) continue;  // the whole segment has no outer partner
    const T wsT = (T)ws;
    if (nb1) {
      for (int i = lane; i < d.hist_f + d.hist_i; i += 32) hf[i] = 0.f;  // hi follows hf
      __syncwarp();
    }
    unsigned int obits = 0;
    if (d.nfam && d.nob) {  // predicates on outer relations, once per segment
      unsigned int mine = 0;
      if (lane < d.nob) {
        const DOuter &o = d.outer[d.obit_outer[lane]];
        int64_t ok = 0;
        for (int i = 0; i < d.seg.ndig; ++i)
          if (o.dstride[i]) ok += ((int64_t)wk.seg / d.seg.radix[i]) % d.seg.dom[i] * o.dstride[i];
        if (__ldg(o.v.v64 + ok * o.v.ncols + d.obit_col[lane]) > 0.0) mine = 1u << d.obit_pos[lane];
      }
      obits = __reduce_or_sync(0xffffffffu, mine);
    }
    T acc[NM][W];
#pragma unroll
    for (int j = 0; j < NM; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[j][w] = T(0);
    const long long rend = wk.r0 + wk.len;
    int kn[RU];
    T xn[RU][FMAXX];
    auto load = [&](long long rb, int (&kk)[RU], T (&xv)[RU][FMAXX]) {
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const long long r = rb + 32 * u;
        const bool ok = r < rend;
        int k = 0;
        if (ok && d.ni) {
          k = ldi(d.col[d.kslot[0]], r) * (int)d.kstride[0];
          if (d.nk > 1) k += ldi(d.col[d.kslot[1]], r) * (int)d.kstride[1];
        }
        kk[u] = ok ? k : -1;
#pragma unroll
        for (int i = 0; i < FMAXX; ++i) xv[u][i] = (ok && i < nx) ? ldn<T>(d.col[d.xslot[i]], r) : T(0);
      }
    };
    load(wk.r0 + lane, kn, xn);
    for (long long rb = wk.r0 + lane; rb < rend; rb += 32 * RU) {
      int kk[RU];
      T xv[RU][FMAXX];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        kk[u] = kn[u];
#pragma unroll
        for (int i = 0; i < FMAXX; ++i) xv[u][i] = xn[u][i];
      }
      if (rb + 32 * RU < rend) load(rb + 32 * RU, kn, xn);  // prefetch the next step
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const int k = kk[u];
        if (k < 0) continue;
        const long long r = rb + 32 * u;
        T v[W];
        if (d.ni) {
#pragma unroll
          for (int w = 0; w < W; ++w) v[w] = (w < nw) ? table[(int64_t)k * nw + w] : T(0);
        } else {
          v[0] = T(1);
#pragma unroll
          for (int w = 1; w < W; ++w) v[w] = T(0);
        }
        if (v[0] == T(0)) continue;  // no partner in the inner relation: not in the join
        T m[NM];
#pragma unroll
        for (int j = 0; j < NM; ++j) {
          T p = T(1);
#pragma unroll
          for (int i = 0; i < FMAXX; ++i)
            if (i < nx) {
              const int e = d.mexp[j][i];
              if (e) p *= powu<T>(xv[u][i], e);
            }
          m[j] = p;
        }
        for (int f = 0; f < nind; ++f) {
          const DFac fc = sd.ind[f];
          if (!pred(d.col[fc.col], r, fc.op, fc.t)) {
            const int jm = sd.ind_mono[f];
#pragma unroll
            for (int j = 0; j < NM; ++j)
              if (j == jm) m[j] = T(0);
          }
        }
#pragma unroll
        for (int j = 0; j < NM; ++j)
#pragma unroll
          for (int w = 0; w < W; ++w) acc[j][w] += m[j] * v[w];
        int leaf = -1;
        if (d.nfam) {  // the filter of the family this tuple satisfies (filters are disjoint)
          unsigned int bits = obits;
          if (d.ibit_code >= 0) bits |= (unsigned int)codes[(int64_t)k * ncode + d.ibit_code];
          for (int q = 0; q < d.nrb; ++q)
            if (pred(d.col[d.rb[q].col], r, d.rb[q].op, d.rb[q].t)) bits |= 1u << d.rb_pos[q];
          for (int f = 0; f < d.nfam; ++f)
            if ((bits & d.fmask[f]) == d.fmask[f]) { leaf = f; break; }
        }
        for (int s = 0; s < nb1; ++s) {
          const DFastB1 &b = sd.b1[s];
          int g = 0;
          bool ok = true;
          for (int i = 0; i < b.nref; ++i) {
            const DGroupRef &q = b.ref[i];
            int code = (q.src == 3) ? codes[(int64_t)k * ncode + q.b]
                       : (q.src == 4) ? leaf
                                      : row_code(d.col[q.a], r, q.kind, d.thr + q.thr0, q.nthr);
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
        const int lsplit = d.b3leaf;
        for (int c = 0; c < n3 && (lsplit == 1 || leaf >= 0); ++c) {
          T val = sel<NM, T>(m, sd.j3[c]);
          if (val == T(0)) continue;
          const int pc = sd.p3col[c] * lsplit + (lsplit > 1 ? leaf : 0);
          if (sd.int3[c]) {
            unsigned long long iv = (unsigned long long)val * ws;
            if (d.smem_p) atomicAdd(Pi + (int64_t)k * n3i * lsplit + pc, (unsigned int)iv);
            else atomicAdd(d.p3i + (int64_t)k * n3i * lsplit + pc, iv);
          } else {
            val *= wsT;
            if (d.smem_p) atomicAdd(Pf + (int64_t)k * n3f * lsplit + pc, val);
            else if (sizeof(T) == 8) atomicAdd(d.p3f + (int64_t)k * n3f * lsplit + pc, (double)val);
            else atomicAdd(d.p3f32 + (int64_t)k * n3f * lsplit + pc, (float)val);
          }
        }
        // CTA-private accumulation (no outer dependency): items of every filter, then the
        // items of this tuple's filter
        const int b4a = d.nb4 ? d.b4_off[0] : 0, b4b = d.nb4 ? d.b4_off[1] : 0;
        const int b4c = (d.nb4 && leaf >= 0) ? d.b4_off[leaf + 1] : 0, b4d = (d.nb4 && leaf >= 0) ? d.b4_off[leaf + 2] : 0;
        for (int ii = b4a; ii < b4b + (b4d - b4c); ++ii) {
          const int i = ii < b4b ? ii : b4c + (ii - b4b);
          T val = sel<NM, T>(m, d.b4_j[i]) * sel<W, T>(v, d.b4_w[i]);
          if (val == T(0)) continue;
          int64_t cell = 0;
          bool okc = true;
          for (int g = d.b4_g0[i]; g < d.b4_g0[i] + d.b4_ng[i]; ++g) {
            const DGroupRef q = d.grefs4[g];
            int code = (q.src == 3) ? codes[(int64_t)k * ncode + q.b]
                                    : row_code(d.col[q.a], r, q.kind, d.thr + q.thr0, q.nthr);
            if (code < 0) okc = false;
            cell += (int64_t)code * q.stride;
          }
          if (!okc) continue;
          if (d.b4_int[i]) atomicAdd(b4i + d.b4_so[i] + cell * d.b4_cellmul[i], (unsigned int)val * (unsigned int)ws);
          else atomicAdd(b4f + d.b4_so[i] + cell * d.b4_cellmul[i], val * wsT);
        }
      }
    }
    // segment sums: warp reduction, one atomic per entry spread over the lanes
    const int n0 = d.nm * nw;
    T ival = T(0);
    const int my_ij = lane < d.n0i ? d.i0j[lane] : -1, my_iw = lane < d.n0i ? d.i0w[lane] : -1;
#pragma unroll
    for (int j = 0; j < NM; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) {
        if (j < d.nm && w < nw) {
          T t = acc[j][w];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (lane == ((j * W + w) & 31) && t != T(0))
            atomicAdd(reinterpret_cast<T *>(d.phi0f) + (int64_t)wk.seg * n0 + j * nw + w, t);
          if (j == my_ij && w == my_iw) ival = t;
        }
      }
    if (lane < d.n0i) {
      unsigned long long it = (unsigned long long)(ival + T(0.5));
      if (it) atomicAdd(d.phi0i + (int64_t)wk.seg * d.n0i + lane, it);
    }
    if (nb1) {
      __syncwarp();
      for (int s = 0; s < nb1; ++s) {
        const DFastB1 &b = sd.b1[s];
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
    for (int64_t i = tid; i < d.nkeys * n3f * d.b3leaf; i += bs)
      if (Pf[i] != T(0)) atomicAdd(d.p3f + i, (double)Pf[i]);
    for (int64_t i = tid; i < d.nkeys * n3i * d.b3leaf; i += bs)
      if (Pi[i]) atomicAdd(d.p3i + i, (unsigned long long)Pi[i]);
  }
  if (d.nb4mirror) {
    __syncthreads();
    for (int mm = 0; mm < d.nb4mirror; ++mm) {
      const DMirror mr = d.b4mirror[mm];
      for (int i = tid; i < mr.len; i += bs) {
        if (mr.integral) { if (b4i[mr.soff + i]) atomicAdd(d.icnt + mr.gout + i, (unsigned long long)b4i[mr.soff + i]); }
        else if (b4f[mr.soff + i] != T(0)) atomicAdd(d.fsum + mr.gout + i, (double)b4f[mr.soff + i]);
      }
    }
  }
}


// Lean root pass: the same outputs as fast_pass_kernel for batches whose root-level
// monomials are the degree <= 2 basis over NX value columns, whose grouped per-segment sums
// are inner COUNTs and whose root-to-inner partials read basis monomials. Straight-line
// per-tuple code (no descriptor loops): loads of the next step are in flight while the
// current one is processed.
template <int NX>
struct Basis { static constexpr int N = 1 + NX + NX * (NX + 1) / 2; };

template <typename T, int NX>
__device__ __forceinline__ void basis(const T (&x)[NX > 0 ? NX : 1], T (&u)[Basis<NX>::N]) {
  u[0] = T(1);
#pragma unroll
  for (int i = 0; i < NX; ++i) u[1 + i] = x[i];
  int q = 1 + NX;
#pragma unroll
  for (int i = 0; i < NX; ++i)
#pragma unroll
    for (int j = i; j < NX; ++j) u[q++] = x[i] * x[j];
}

// 4 consecutive values of a column at tuple 4q (the column is padded past its end)
template <typename T>
__device__ __forceinline__ void load4(const DCol &c, int64_t q, T (&o)[4]) {
  if (c.dtype == LMFAO_F32) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(c.p) + q);
    o[0] = (T)v.x; o[1] = (T)v.y; o[2] = (T)v.z; o[3] = (T)v.w;
  } else if (c.dtype == LMFAO_U8) {
    const unsigned int v = __ldg(reinterpret_cast<const unsigned int *>(c.p) + q);
    o[0] = (T)(v & 0xffu); o[1] = (T)((v >> 8) & 0xffu); o[2] = (T)((v >> 16) & 0xffu); o[3] = (T)(v >> 24);
  } else {
    const int4 v = __ldg(reinterpret_cast<const int4 *>(c.p) + q);
    o[0] = (T)v.x; o[1] = (T)v.y; o[2] = (T)v.z; o[3] = (T)v.w;
  }
}

template <typename T, int NX, int W, bool VEC>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512, 1) lean_pass_kernel(DFast d) {
  constexpr int NM = Basis<NX>::N;
  constexpr int XA = NX > 0 ? NX : 1;
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = bs >> 5;
  size_t off = 0;
  T *Pf = reinterpret_cast<T *>(smem);
  unsigned int *Pi = nullptr;
  if (d.smem_p) {
    off += sizeof(T) * (size_t)d.nkeys * d.n3f;
    Pi = reinterpret_cast<unsigned int *>(smem + off);
    off += 4 * (size_t)d.nkeys * d.n3i;
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
  unsigned int *hi = reinterpret_cast<unsigned int *>(smem + off) + (size_t)warp * d.hist_i;
  if (d.smem_p) {
    for (int64_t i = tid; i < d.nkeys * d.n3f; i += bs) Pf[i] = T(0);
    for (int64_t i = tid; i < d.nkeys * d.n3i; i += bs) Pi[i] = 0u;
  }
  __syncthreads();
  const int nb1 = d.nb1, n3 = d.n3, nw = d.nw, ncode = d.ncode, n3f = d.n3f, n3i = d.n3i;
  const DCol kc = d.col[d.kslot[0]];
  DCol xc[XA];
#pragma unroll
  for (int i = 0; i < XA; ++i) xc[i] = d.col[d.xslot[i]];

  for (;;) {
    int64_t wi = 0;
    if (lane == 0) wi = atomicAdd(d.ticket, 1u);
    wi = __shfl_sync(0xffffffffu, wi, 0);
    if (wi >= d.nwork) break;
    const DWork wk = d.work[wi];
    const unsigned long long ws = d.wseg[wk.seg];
    if (ws == 0) continue;  // the whole segment has no outer partner
    const T wsT = (T)ws;
    if (nb1) {
      for (int i = lane; i < d.hist_i; i += 32) hi[i] = 0u;
      __syncwarp();
    }
    T acc[NM][W];
#pragma unroll
    for (int j = 0; j < NM; ++j)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[j][w] = T(0);
    const long long rend = wk.r0 + wk.len;
    auto one = [&](const int k, const T (&xt)[XA]) {
      T v[W];
      if (d.ni) {
#pragma unroll
        for (int w = 0; w < W; ++w) v[w] = (w < nw) ? table[k * nw + w] : T(0);
      } else {
        v[0] = T(1);
#pragma unroll
        for (int w = 1; w < W; ++w) v[w] = T(0);
      }
      if (v[0] == T(0)) return;  // no partner in the inner relation: not in the join
      T um[NM];
      basis<T, NX>(xt, um);
#pragma unroll
      for (int j = 0; j < NM; ++j)
#pragma unroll
        for (int w = 0; w < W; ++w) acc[j][w] += um[j] * v[w];
      const unsigned int cnt = (unsigned int)v[0];
#pragma unroll
      for (int s = 0; s < FMAXB1; ++s)
        if (s < nb1) {
          const int code = codes[k * ncode + d.b1code[s]];
          if (code >= 0) atomicAdd(hi + d.b1[s].smem_i + code, cnt);
        }
#pragma unroll
      for (int c = 0; c < FMAXC; ++c)
        if (c < n3) {
          const int pc = d.p3col[c];
          if (d.int3[c]) {
            if (d.smem_p) atomicAdd(Pi + k * n3i + pc, (unsigned int)ws);
            else atomicAdd(d.p3i + (int64_t)k * n3i + pc, ws);
          } else {
            const T val = wsT * sel<NM, T>(um, d.j3[c]);
            if (d.smem_p) atomicAdd(Pf + k * n3f + pc, val);
            else if (sizeof(T) == 8) atomicAdd(d.p3f + (int64_t)k * n3f + pc, (double)val);
            else atomicAdd(d.p3f32 + (int64_t)k * n3f + pc, (float)val);
          }
        }
    };
    if (VEC) {
      // quads of 4 consecutive tuples per lane; the quad of the next step is in flight
      const int64_t qa = wk.r0 >> 2, qe = (rend + 3) >> 2;
      int kq[4];
      T xq[XA][4];
      auto loadq = [&](int64_t q, int (&kk)[4], T (&xx)[XA][4]) {
        if (q >= qe) return;
        if (d.ni) {
          const int4 v = __ldg(reinterpret_cast<const int4 *>(kc.p) + q);
          kk[0] = v.x; kk[1] = v.y; kk[2] = v.z; kk[3] = v.w;
        } else {
          kk[0] = kk[1] = kk[2] = kk[3] = 0;
        }
#pragma unroll
        for (int i = 0; i < XA; ++i)
          if (NX > 0) load4<T>(xc[i], q, xx[i]);
      };
      loadq(qa + lane, kq, xq);
      for (int64_t q = qa + lane; q < qe; q += 32) {
        int kk[4];
        T xx[XA][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          kk[u] = kq[u];
#pragma unroll
          for (int i = 0; i < XA; ++i) xx[i][u] = xq[i][u];
        }
        loadq(q + 32, kq, xq);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long r = 4 * q + u;
          if (r < wk.r0 || r >= rend) continue;
          T xt[XA];
#pragma unroll
          for (int i = 0; i < XA; ++i) xt[i] = NX > 0 ? xx[i][u] : T(0);
          one(kk[u], xt);
        }
      }
    } else {
      int kn[RU];
      T xn[RU][XA];
#pragma unroll
      for (int u = 0; u < RU; ++u) {
        const long long r = wk.r0 + lane + 32 * u;
        const bool ok = r < rend;
        kn[u] = ok ? (d.ni ? ldi(kc, r) : 0) : -1;
#pragma unroll
        for (int i = 0; i < XA; ++i) xn[u][i] = (ok && NX > 0) ? ldn<T>(xc[i], r) : T(0);
      }
      for (long long rb = wk.r0 + lane; rb < rend; rb += 32 * RU) {
        int kk[RU];
        T xv[RU][XA];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
          kk[u] = kn[u];
#pragma unroll
          for (int i = 0; i < XA; ++i) xv[u][i] = xn[u][i];
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {  // prefetch the next step
          const long long r = rb + 32 * (RU + u);
          const bool ok = r < rend;
          kn[u] = ok ? (d.ni ? ldi(kc, r) : 0) : -1;
#pragma unroll
          for (int i = 0; i < XA; ++i) xn[u][i] = (ok && NX > 0) ? ldn<T>(xc[i], r) : T(0);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
          if (kk[u] >= 0) one(kk[u], xv[u]);
      }
    }
    // segment sums: reduce-scatter over the warp by recursive halving; lane L ends with
    // the totals of the flat entries [L*F, L*F + F) of acc (entry j*W + w)
    constexpr int V = NM * W, F = (V + 31) / 32, PV = 32 * F;
    T r[PV];
#pragma unroll
    for (int i = 0; i < PV; ++i) r[i] = i < V ? acc[i / W][i % W] : T(0);
#pragma unroll
    for (int lvl = 0; lvl < 5; ++lvl) {
      const int o = 16 >> lvl, h = PV >> (lvl + 1);
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const T send = up ? r[i] : r[i + h];
        const T keep = up ? r[i + h] : r[i];
        r[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    const int n0 = NM * nw;
#pragma unroll
    for (int e = 0; e < F; ++e) {
      const int i = lane * F + e, j = i / W, w = i - j * W;
      if (i < V && w < nw && r[e] != T(0))
        atomicAdd(reinterpret_cast<T *>(d.phi0f) + (int64_t)wk.seg * n0 + j * nw + w, r[e]);
    }
    // integral segment sums (exact small integers carried in T) to their lanes
    T ival = T(0);
    const int q = lane < d.n0i ? d.i0j[lane] * W + d.i0w[lane] : 0;
#pragma unroll
    for (int e = 0; e < F; ++e) {
      const T t = __shfl_sync(0xffffffffu, r[e], q / F);
      if (e == q % F) ival = t;
    }
    if (lane < d.n0i) {
      unsigned long long it = (unsigned long long)(ival + T(0.5));
      if (it) atomicAdd(d.phi0i + (int64_t)wk.seg * d.n0i + lane, it);
    }
    if (nb1) {
      __syncwarp();
      for (int s = 0; s < nb1; ++s) {
        const int G = d.b1[s].G, so = d.b1[s].smem_i;
        const int64_t gb = (int64_t)wk.seg * d.phi1i_seg + d.b1[s].gbase_i;
        for (int i = lane; i < G; i += 32) {
          unsigned int x = hi[so + i];
          if (x) atomicAdd(d.phi1i + gb + i, x);
        }
      }
      __syncwarp();
    }
  }
  if (d.smem_p) {
    __syncthreads();
    for (int64_t i = tid; i < d.nkeys * n3f; i += bs)
      if (Pf[i] != T(0)) atomicAdd(d.p3f + i, (double)Pf[i]);
    for (int64_t i = tid; i < d.nkeys * n3i; i += bs)
      if (Pi[i]) atomicAdd(d.p3i + i, (unsigned long long)Pi[i]);
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
      unsigned long long p = d.p3i[k * d.n3i + item.c];
      if (p) atomicAdd(d.icnt + item.out + cell * item.cellmul, p * (unsigned long long)vv);
    } else {
      double p = item.pint ? (double)d.p3i[k * d.n3i + item.c]
                 : d.p3f32   ? (double)d.p3f32[k * d.n3f + item.c]
                             : d.p3f[k * d.n3f + item.c];
      if (p != 0.0) atomicAdd(d.fsum + item.out + cell * item.cellmul, p * vv);
    }
  }
}

}  // namespace

void launch_fast_prep(const DFast &d, const double *v64, int vcols, const int *wcol, const int32_t *vcodes,
                      int vncodes, const int *codecol, void *table, int *codes, bool fp64, cudaStream_t s,
                      const int2 *ib, int nib) {
  if (!d.ni || d.nkeys == 0) return;
  int grid = (int)std::min<int64_t>((d.nkeys + 255) / 256, 148 * 8);
  if (fp64)
    fast_prep_kernel<double><<<grid, 256, 0, s>>>(d.nkeys, v64, vcols, wcol, d.nw, (double *)table, vcodes, vncodes,
                                                   codecol, d.ncode, codes, ib, nib, d.ibit_code);
  else
    fast_prep_kernel<float><<<grid, 256, 0, s>>>(d.nkeys, v64, vcols, wcol, d.nw, (float *)table, vcodes, vncodes,
                                                  codecol, d.ncode, codes, ib, nib, d.ibit_code);
}

size_t fast_smem(const DFast &d, bool fp64, int block) {
  size_t ts = fp64 ? 8 : 4;
  size_t off = 0;
  const size_t ls = d.b3leaf > 0 ? (size_t)d.b3leaf : 1;
  if (d.smem_p) off += ts * (size_t)d.nkeys * d.n3f * ls + 4 * (size_t)d.nkeys * d.n3i * ls;
  off = (off + 15) & ~(size_t)15;
  if (d.smem_view && d.ni) off += ts * (size_t)d.nkeys * d.nw + 4 * (size_t)d.nkeys * d.ncode;
  off = (off + 15) & ~(size_t)15;
  off += (size_t)(block / 32) * (d.hist_f + d.hist_i) * 4;
  off = (off + 15) & ~(size_t)15;
  off += ts * (size_t)d.b4_fcells;
  off = (off + 15) & ~(size_t)15;
  off += 4 * (size_t)d.b4_icells;
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

bool lean_shape_ok(int nx, int nw) { return nx >= 0 && nx <= 3 && nw >= 1 && nw <= 8; }

template <typename T, int NX, int W>
static void go_lean(const DFast &d, int grid, int block, size_t smem, cudaStream_t s) {
  if (d.vec) {
    cudaFuncSetAttribute(lean_pass_kernel<T, NX, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    lean_pass_kernel<T, NX, W, true><<<grid, block, smem, s>>>(d);
  } else {
    cudaFuncSetAttribute(lean_pass_kernel<T, NX, W, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    lean_pass_kernel<T, NX, W, false><<<grid, block, smem, s>>>(d);
  }
}

template <typename T, int NX>
static void lean_w(const DFast &d, int grid, int block, size_t smem, cudaStream_t s) {
  if (d.nw <= 1) go_lean<T, NX, 1>(d, grid, block, smem, s);
  else if (d.nw <= 2) go_lean<T, NX, 2>(d, grid, block, smem, s);
  else if (d.nw <= 4) go_lean<T, NX, 4>(d, grid, block, smem, s);
  else if (d.nw <= 6) go_lean<T, NX, 6>(d, grid, block, smem, s);
  else go_lean<T, NX, 8>(d, grid, block, smem, s);
}

template <typename T>
static void lean_x(const DFast &d, int grid, int block, size_t smem, cudaStream_t s) {
  switch (d.nx) {
    case 0: lean_w<T, 0>(d, grid, block, smem, s); break;
    case 1: lean_w<T, 1>(d, grid, block, smem, s); break;
    case 2: lean_w<T, 2>(d, grid, block, smem, s); break;
    default: lean_w<T, 3>(d, grid, block, smem, s); break;
  }
}

bool launch_fast_pass(const DFast &d, bool fp64, int grid, int block, cudaStream_t s) {
  size_t smem = fast_smem(d, fp64, block);
  if (d.lean) {
    if (fp64) lean_x<double>(d, grid, block, smem, s);
    else lean_x<float>(d, grid, block, smem, s);
    return true;
  }
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
