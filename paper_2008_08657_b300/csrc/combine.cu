// The combine of the root group: every output entry is
//     out[ocell(s) + icell] += SUM over segments s of psi_t(s) * Y_c(s)
// where psi_t is a product of outer view columns (and segment-key factors) and Y_c one
// per-segment sum (PHI0 column, or PHI1 column at a fixed inner group code).
//
// The segments of one CTA form a contiguous range of the segment key, so outer group
// cells (codes of outer views keyed by a prefix of the segment key) change rarely: each
// thread owns up to EMAX entries, accumulates them in registers and writes an entry's
// sum out only when its outer cell changes (or at the end). Per tile of segments the
// outer view rows are staged once in shared memory, then every distinct psi_t, then the
// Y rows; FP32 (or FP64) products and partial sums, FP64 / INT64 output reduction.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lmfao {

namespace {

__device__ __forceinline__ int64_t digit(const DSegment &s, int64_t seg, int i) { return (seg / s.radix[i]) % s.dom[i]; }

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

template <typename T, int EMAX>
__global__ void __launch_bounds__(512) combine2_kernel(DComb2 d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = blockDim.x, tid = threadIdx.x, TS = d.tile;
  // shared layout (8-byte arrays first)
  long long *keys = reinterpret_cast<long long *>(smem);                     // TS x nouter
  long long *ocell = keys + (size_t)TS * d.nouter;                          // TS x nog
  unsigned long long *psii = reinterpret_cast<unsigned long long *>(ocell + (size_t)TS * d.nog);  // TS x npsi
  unsigned long long *yi = psii + (size_t)TS * d.npsi;                      // TS x nyi
  unsigned long long *mi = yi + (size_t)TS * d.nyi;                         // mirror (integral)
  T *stage = reinterpret_cast<T *>(mi + d.mirror_i);                        // TS x nstage
  T *psif = stage + (size_t)TS * d.nstage;                                  // TS x npsi
  T *yf = psif + (size_t)TS * d.npsi;                                       // TS x nyf
  T *mf = yf + (size_t)TS * d.nyf;                                          // mirror (float)

  for (int i = tid; i < d.mirror_i; i += bs) mi[i] = 0ull;
  for (int i = tid; i < d.mirror_f; i += bs) mf[i] = T(0);

  // entries owned by this thread (chunk blockIdx.y)
  const int ebase = blockIdx.y * bs * EMAX;
  int epsi[EMAX], ey[EMAX], eog[EMAX], eint[EMAX], eyi[EMAX], cur[EMAX];
  T accf[EMAX];
  unsigned long long acci[EMAX];
#pragma unroll
  for (int k = 0; k < EMAX; ++k) {
    int e = ebase + tid + k * bs;
    if (e < d.nent) {
      const DEntry en = d.ent[e];
      epsi[k] = en.psi;
      ey[k] = en.ycol;
      eog[k] = en.og;
      eint[k] = en.integral;
      eyi[k] = en.yint;
    } else {
      epsi[k] = -1;
      ey[k] = eog[k] = eint[k] = eyi[k] = 0;
    }
    cur[k] = -1;
    accf[k] = T(0);
    acci[k] = 0ull;
  }

  auto flush = [&](int k) {
    if (cur[k] < 0) return;
    const int e = ebase + tid + k * bs;
    const DEntry en = d.ent[e];
    const long long idx = en.out + ((long long)cur[k] + en.icell) * en.cellmul;
    if (eint[k]) {
      if (acci[k]) {
        if (en.so >= 0) atomicAdd(mi + en.so + ((long long)cur[k] + en.icell) * en.cellmul, acci[k]);
        else atomicAdd(d.icnt + idx, acci[k]);
      }
      acci[k] = 0ull;
    } else {
      if (accf[k] != T(0)) {
        if (en.so >= 0) atomicAdd(mf + en.so + ((long long)cur[k] + en.icell) * en.cellmul, accf[k]);
        else atomicAdd(d.fsum + idx, (double)accf[k]);
      }
      accf[k] = T(0);
    }
  };

  // contiguous segment range of this CTA
  const int64_t per = (d.nseg + gridDim.x - 1) / gridDim.x;
  const int64_t sbeg = (int64_t)blockIdx.x * per;
  const int64_t send = min(d.nseg, sbeg + per);
  for (int64_t seg0 = sbeg; seg0 < send; seg0 += TS) {
    const int nt = (int)min((int64_t)TS, send - seg0);
    __syncthreads();
    // 1. outer view keys of each segment (-1: no outer partner)
    for (int idx = tid; idx < nt * d.nouter; idx += bs) {
      int s = idx / d.nouter, o = idx - s * d.nouter;
      int64_t seg = seg0 + s;
      long long k = -1;
      if (d.wseg[seg]) {
        k = 0;
        for (int i = 0; i < d.seg.ndig; ++i)
          if (d.outer[o].dstride[i]) k += digit(d.seg, seg, i) * d.outer[o].dstride[i];
      }
      keys[idx] = k;
    }
    // Y rows of the tile
    for (int idx = tid; idx < nt * d.nyf; idx += bs) {
      int s = idx / d.nyf, j = idx - s * d.nyf;
      int64_t seg = seg0 + s;
      yf[idx] = j < d.n0f ? reinterpret_cast<const T *>(d.phi0f)[seg * d.n0f + j]
                          : (T)d.phi1f[seg * d.phi1f_seg + (j - d.n0f)];
    }
    for (int idx = tid; idx < nt * d.nyi; idx += bs) {
      int s = idx / d.nyi, j = idx - s * d.nyi;
      int64_t seg = seg0 + s;
      yi[idx] = j < d.n0i ? d.phi0i[seg * d.n0i + j] : (unsigned long long)d.phi1i[seg * d.phi1i_seg + (j - d.n0i)];
    }
    __syncthreads();
    // 2. staged outer view columns and outer cells
    for (int idx = tid; idx < nt * d.nstage; idx += bs) {
      int s = idx / d.nstage, j = idx - s * d.nstage;
      int2 sc = d.stage_col[j];  // (outer view, column)
      long long k = keys[s * d.nouter + sc.x];
      stage[idx] = k < 0 ? T(0) : (T)__ldg(d.outer[sc.x].v.v64 + k * d.outer[sc.x].v.ncols + sc.y);
    }
    for (int idx = tid; idx < nt * d.nog; idx += bs) {
      int s = idx / d.nog, g = idx - s * d.nog;
      int64_t seg = seg0 + s;
      long long cell = d.wseg[seg] ? 0 : -1;
      for (int r = d.og_off[g]; r < d.og_off[g + 1] && cell >= 0; ++r) {
        DGroupRef q = d.grefs[r];
        long long code;
        if (q.src == 0) code = digit(d.seg, seg, q.a);
        else {
          long long k = keys[s * d.nouter + q.a];
          code = k < 0 ? -1 : __ldg(d.outer[q.a].v.codes + k * d.outer[q.a].v.ncodes + q.b);
        }
        if (code < 0) cell = -1;
        else cell += code * q.stride;
      }
      ocell[idx] = cell;
    }
    __syncthreads();
    // 3. outer terms
    for (int idx = tid; idx < nt * d.npsi; idx += bs) {
      int s = idx / d.npsi, t = idx - s * d.npsi;
      int64_t seg = seg0 + s;
      const DPsi p = d.psi[t];
      T v = T(1);
      unsigned long long iv = 1ull;
      for (int f = p.f0; f < p.f0 + p.nf; ++f) {
        DSegFac q = d.segfacs[f];
        int64_t dg = digit(d.seg, seg, q.digit);
        if (q.ind) {
          if (!cmpx<double>((double)dg, (double)q.t, q.op)) { v = T(0); iv = 0; }
        } else {
          T x = (T)dg, y = x;
          for (int e = 1; e < q.pow; ++e) y *= x;
          v *= y;
          iv *= (unsigned long long)dg;  // unused for integral terms (no value factors)
        }
      }
      for (int i = p.p0; i < p.p0 + p.np; ++i) {
        T x = stage[s * d.nstage + d.psi_stage[i]];
        v *= x;
        iv *= (unsigned long long)x;
      }
      psif[idx] = v;
      psii[idx] = p.integral ? iv : 0ull;
    }
    __syncthreads();
    // 4. entries
#pragma unroll
    for (int k = 0; k < EMAX; ++k) {
      if (epsi[k] < 0) continue;
      for (int s = 0; s < nt; ++s) {
        const long long cell = ocell[s * d.nog + eog[k]];
        if (cell < 0) continue;
        if (cell != cur[k]) {
          flush(k);
          cur[k] = (int)cell;
        }
        if (eint[k]) acci[k] += psii[s * d.npsi + epsi[k]] * yi[s * d.nyi + ey[k]];
        else if (eyi[k]) accf[k] += psif[s * d.npsi + epsi[k]] * (T)yi[s * d.nyi + ey[k]];
        else accf[k] += psif[s * d.npsi + epsi[k]] * yf[s * d.nyf + ey[k]];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < EMAX; ++k)
    if (epsi[k] >= 0) flush(k);
  __syncthreads();
  for (int m = 0; m < d.nmirror; ++m) {
    DMirror mr = d.mirror[m];
    for (int i = tid; i < mr.len; i += bs) {
      if (mr.integral) { if (mi[mr.soff + i]) atomicAdd(d.icnt + mr.gout + i, mi[mr.soff + i]); }
      else if (mf[mr.soff + i] != T(0)) atomicAdd(d.fsum + mr.gout + i, (double)mf[mr.soff + i]);
    }
  }
}

}  // namespace

size_t combine2_smem(const DComb2 &d, bool fp64) {
  size_t ts = fp64 ? 8 : 4;
  size_t b = 8 * ((size_t)d.tile * (d.nouter + d.nog + d.npsi + d.nyi) + d.mirror_i);
  b += ts * ((size_t)d.tile * (d.nstage + d.npsi + d.nyf) + d.mirror_f);
  return b;
}

int combine2_emax(int nent, int block) {
  int per = (nent + block - 1) / block;
  if (per <= 2) return 2;
  if (per <= 4) return 4;
  return 8;
}

void launch_combine2(const DComb2 &d, bool fp64, int grid, int block, cudaStream_t s) {
  size_t smem = combine2_smem(d, fp64);
  int emax = combine2_emax(d.nent, block);
  int chunks = (d.nent + block * emax - 1) / (block * emax);
  dim3 g(grid, chunks < 1 ? 1 : chunks);
#define LMFAO_C2(TT, E)                                                                               \
  {                                                                                                   \
    cudaFuncSetAttribute(combine2_kernel<TT, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    combine2_kernel<TT, E><<<g, block, smem, s>>>(d);                                                 \
  }
  if (fp64) {
    if (emax == 2) LMFAO_C2(double, 2) else if (emax == 4) LMFAO_C2(double, 4) else LMFAO_C2(double, 8)
  } else {
    if (emax == 2) LMFAO_C2(float, 2) else if (emax == 4) LMFAO_C2(float, 4) else LMFAO_C2(float, 8)
  }
#undef LMFAO_C2
}

}  // namespace lmfao
