// Prefix-block combine (see DComb3 in kernels.cuh).
//
// Per block p of m segments (one value of the segment-key prefix):
//   1. stage the B-view columns of the m segments and their Y rows (per-segment sums),
//   2. B terms b_beta(s) (products of staged columns and minor-digit factors),
//   3. Z_p[beta][c] = SUM_s b_beta(s) Y_c(s) for every (beta, c)  -- FP32 (or FP64),
//      exact INT64 for integral B terms x integral Y columns,
//   4. A terms a_alpha(p) from the A-view rows of the prefix and the outer cells,
//   5. every entry owned by a thread: acc += a_alpha(p) * Z_p[beta][c], written out when
//      its outer cell changes (outer cells are constant inside a block).
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lmfao {

namespace {

__device__ __forceinline__ int64_t digit3(const DSegment &s, int64_t seg, int i) { return (seg / s.radix[i]) % s.dom[i]; }

template <typename X>
__device__ __forceinline__ bool cmp3(X x, X t, int op) {
  switch (op) {
    case LMFAO_LE: return x <= t;
    case LMFAO_LT: return x < t;
    case LMFAO_GE: return x >= t;
    case LMFAO_GT: return x > t;
    case LMFAO_EQ: return x == t;
    default: return x != t;
  }
}

template <typename T>
__device__ __forceinline__ void term3(const DPsi &p, const DSegFac *sf, const int *part, const T *staged,
                                      const DSegment &sg, int64_t seg, T &v, unsigned long long &iv) {
  v = T(1);
  iv = 1ull;
  for (int f = p.f0; f < p.f0 + p.nf; ++f) {
    DSegFac q = sf[f];
    int64_t dg = digit3(sg, seg, q.digit);
    if (q.ind) {
      if (!cmp3<double>((double)dg, (double)q.t, q.op)) { v = T(0); iv = 0; }
    } else {
      T x = (T)dg, y = x;
      for (int e = 1; e < q.pow; ++e) y *= x;
      v *= y;
    }
  }
  for (int i = p.p0; i < p.p0 + p.np; ++i) {
    T x = staged[part[i]];
    v *= x;
    iv *= (unsigned long long)x;
  }
  if (!p.integral) iv = 0ull;
}

template <typename T, int EMAX>
__global__ void __launch_bounds__(512) combine3_kernel(DComb3 d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = blockDim.x, tid = threadIdx.x;
  const int m = (int)d.m, ny = d.nyf + d.nyi;
  // shared layout (8-byte arrays first)
  long long *kmin = reinterpret_cast<long long *>(smem);                    // nouter x m: minor-digit key parts
  unsigned long long *ysi = reinterpret_cast<unsigned long long *>(kmin + (size_t)d.nouter * m);  // m x nyi
  unsigned long long *bti = ysi + (size_t)m * d.nyi;                        // m x nbi
  unsigned long long *zi = bti + (size_t)m * d.nbi;                         // nbi x nyi
  unsigned long long *ati = zi + (size_t)d.nbi * d.nyi;                     // na
  long long *ocell = reinterpret_cast<long long *>(ati + d.na);             // nog
  unsigned long long *mi = reinterpret_cast<unsigned long long *>(ocell + d.nog);  // mirror
  T *ysf = reinterpret_cast<T *>(mi + d.mirror_i);                          // m x ny (all Y as T)
  T *bsv = ysf + (size_t)m * ny;                                            // m x nbst
  T *bt = bsv + (size_t)m * d.nbst;                                         // m x nb
  T *zf = bt + (size_t)m * d.nb;                                            // nb x ny
  T *asv = zf + (size_t)d.nb * ny;                                          // nast
  T *at = asv + d.nast;                                                     // na
  T *mf = at + d.na;                                                        // mirror
  __shared__ long long akey[MAXOUT];
  __shared__ int block_live;
  // view-key contribution of the minor digits of the j-th segment of any block (a block is
  // m consecutive segments starting at a multiple of m, so these digits depend on j alone)
  for (int idx = tid; idx < d.nouter * m; idx += bs) {
    const int o = idx / m, j = idx - o * m;
    long long k = 0;
    for (int i = 0; i < d.seg.ndig; ++i)
      if (d.outer[o].dstride[i] && d.seg.radix[i] < d.m) k += ((j / d.seg.radix[i]) % d.seg.dom[i]) * d.outer[o].dstride[i];
    kmin[idx] = k;
  }

  for (int i = tid; i < d.mirror_i; i += bs) mi[i] = 0ull;
  for (int i = tid; i < d.mirror_f; i += bs) mf[i] = T(0);

  const int ebase = blockIdx.y * bs * EMAX;
  int ea[EMAX], eb[EMAX], ec[EMAX], eyi[EMAX], eint[EMAX], eog[EMAX], cur[EMAX];
  T accf[EMAX];
  unsigned long long acci[EMAX];
#pragma unroll
  for (int k = 0; k < EMAX; ++k) {
    int e = ebase + tid + k * bs;
    if (e < d.nent) {
      const DEntry3 en = d.ent[e];
      ea[k] = en.a; eb[k] = en.b; ec[k] = en.c; eyi[k] = en.yint; eint[k] = en.integral; eog[k] = en.og;
    } else {
      ea[k] = -1; eb[k] = ec[k] = eyi[k] = eint[k] = eog[k] = 0;
    }
    cur[k] = -1;
    accf[k] = T(0);
    acci[k] = 0ull;
  }
  auto flush = [&](int k) {
    if (cur[k] < 0) return;
    const DEntry3 en = d.ent[ebase + tid + k * bs];
    const long long rel = ((long long)cur[k] + en.icell) * en.cellmul;
    if (eint[k]) {
      if (acci[k]) {
        if (en.so >= 0) atomicAdd(mi + en.so + rel, acci[k]);
        else atomicAdd(d.icnt + en.out + rel, acci[k]);
      }
      acci[k] = 0ull;
    } else {
      if (accf[k] != T(0)) {
        if (en.so >= 0) atomicAdd(mf + en.so + rel, accf[k]);
        else atomicAdd(d.fsum + en.out + rel, (double)accf[k]);
      }
      accf[k] = T(0);
    }
  };

  const int64_t per = (d.nblocks + gridDim.x - 1) / gridDim.x;
  const int64_t pbeg = (int64_t)blockIdx.x * per, pend = min(d.nblocks, pbeg + per);
  for (int64_t p = pbeg; p < pend; ++p) {
    const int64_t s0 = p * d.m;
    __syncthreads();
    if (tid == 0) block_live = 0;
    __syncthreads();
    // 0. view keys of the block's prefix digits
    if (tid < d.nouter) {
      const DOuter &o = d.outer[tid];
      int64_t k = 0;
      for (int i = 0; i < d.seg.ndig; ++i)
        if (o.dstride[i]) k += digit3(d.seg, s0, i) * o.dstride[i];
      akey[tid] = k;
    }
    __syncthreads();
    // 1. staged B columns and Y rows of the block
    for (int idx = tid; idx < m * d.nbst; idx += bs) {
      int s = idx / d.nbst, j = idx - s * d.nbst;
      int64_t seg = s0 + s;
      T v = T(0);
      if (d.wseg[seg]) {
        block_live = 1;
        int2 sc = d.bstage[j];
        const DOuter &o = d.outer[sc.x];
        const int64_t k = akey[sc.x] + kmin[(size_t)sc.x * m + s];
        v = (T)__ldg(o.v.v64 + k * o.v.ncols + sc.y);
      }
      bsv[idx] = v;
    }
    for (int idx = tid; idx < m * ny; idx += bs) {
      int s = idx / ny, c = idx - s * ny;
      int64_t seg = s0 + s;
      T v;
      if (c < d.nyf) {
        v = c < d.n0f ? reinterpret_cast<const T *>(d.phi0f)[seg * d.n0f + c]
                      : (T)d.phi1f[seg * d.phi1f_seg + (c - d.n0f)];
      } else {
        int ci = c - d.nyf;
        unsigned long long u = ci < d.n0i ? d.phi0i[seg * d.n0i + ci]
                                          : (unsigned long long)d.phi1i[seg * d.phi1i_seg + (ci - d.n0i)];
        ysi[(size_t)s * d.nyi + ci] = u;
        v = (T)u;
      }
      ysf[idx] = v;
    }
    __syncthreads();
    if (!block_live) continue;  // no segment of the block joins its outer views
    // 2. B terms; A-view values of the prefix; outer cells
    for (int idx = tid; idx < m * d.nb; idx += bs) {
      int s = idx / d.nb, b = idx - s * d.nb;
      T v;
      unsigned long long iv;
      term3<T>(d.bterm[b], d.segfacs, d.bpart, bsv + (size_t)s * d.nbst, d.seg, s0 + s, v, iv);
      bt[idx] = v;
      if (b < d.nbi) bti[(size_t)s * d.nbi + b] = iv;
    }
    for (int j = tid; j < d.nast; j += bs) {
      int2 sc = d.astage[j];
      const DOuter &o = d.outer[sc.x];
      asv[j] = (T)__ldg(o.v.v64 + akey[sc.x] * o.v.ncols + sc.y);
    }
    for (int g = tid; g < d.nog; g += bs) {
      long long cell = 0;
      for (int r = d.og_off[g]; r < d.og_off[g + 1] && cell >= 0; ++r) {
        DGroupRef q = d.grefs[r];
        long long code = q.src == 0 ? digit3(d.seg, s0, q.a)
                                    : __ldg(d.outer[q.a].v.codes + akey[q.a] * d.outer[q.a].v.ncodes + q.b);
        if (code < 0) cell = -1;
        else cell += code * q.stride;
      }
      ocell[g] = cell;
    }
    __syncthreads();
    // 3. Z = B^T Y over the block's segments; A terms
    {
      const int nq = (ny + 3) >> 2;  // four Y columns per thread: 5 shared loads per 4 FMA
      for (int o = tid; o < d.nb * nq; o += bs) {
        const int b = o / nq, c0 = 4 * (o - b * nq);
        T z0 = T(0), z1 = T(0), z2 = T(0), z3 = T(0);
        if (c0 + 3 < ny) {
          for (int s = 0; s < m; ++s) {
            const T bv = bt[(size_t)s * d.nb + b];
            const T *y = ysf + (size_t)s * ny + c0;
            z0 += bv * y[0];
            z1 += bv * y[1];
            z2 += bv * y[2];
            z3 += bv * y[3];
          }
        } else {
          for (int s = 0; s < m; ++s) {
            const T bv = bt[(size_t)s * d.nb + b];
            const T *y = ysf + (size_t)s * ny + c0;
            z0 += bv * y[0];
            if (c0 + 1 < ny) z1 += bv * y[1];
            if (c0 + 2 < ny) z2 += bv * y[2];
          }
        }
        T *zo = zf + (size_t)b * ny + c0;
        zo[0] = z0;
        if (c0 + 1 < ny) zo[1] = z1;
        if (c0 + 2 < ny) zo[2] = z2;
        if (c0 + 3 < ny) zo[3] = z3;
      }
    }
    for (int o = tid; o < d.nbi * d.nyi; o += bs) {
      int b = o / d.nyi, c = o - b * d.nyi;
      unsigned long long z = 0;
      for (int s = 0; s < m; ++s) z += bti[(size_t)s * d.nbi + b] * ysi[(size_t)s * d.nyi + c];
      zi[o] = z;
    }
    for (int a = tid; a < d.na; a += bs) {
      T v;
      unsigned long long iv;
      term3<T>(d.aterm[a], d.segfacs, d.apart, asv, d.seg, s0, v, iv);
      at[a] = v;
      ati[a] = iv;
    }
    __syncthreads();
    // 4. entries
#pragma unroll
    for (int k = 0; k < EMAX; ++k) {
      if (ea[k] < 0) continue;
      const long long cell = ocell[eog[k]];
      if (cell < 0) continue;
      if (cell != cur[k]) {
        flush(k);
        cur[k] = (int)cell;
      }
      if (eint[k]) acci[k] += ati[ea[k]] * zi[eb[k] * d.nyi + ec[k]];
      else accf[k] += at[ea[k]] * zf[eb[k] * ny + (eyi[k] ? d.nyf + ec[k] : ec[k])];
    }
  }
#pragma unroll
  for (int k = 0; k < EMAX; ++k)
    if (ea[k] >= 0) flush(k);
  __syncthreads();
  for (int mm = 0; mm < d.nmirror; ++mm) {
    DMirror mr = d.mirror[mm];
    for (int i = tid; i < mr.len; i += bs) {
      if (mr.integral) { if (mi[mr.soff + i]) atomicAdd(d.icnt + mr.gout + i, mi[mr.soff + i]); }
      else if (mf[mr.soff + i] != T(0)) atomicAdd(d.fsum + mr.gout + i, (double)mf[mr.soff + i]);
    }
  }
}

}  // namespace

size_t combine3_smem(const DComb3 &d, bool fp64) {
  size_t ts = fp64 ? 8 : 4;
  const size_t m = (size_t)d.m, ny = (size_t)d.nyf + d.nyi;
  size_t b = 8 * ((size_t)d.nouter * m + m * d.nyi + m * d.nbi + (size_t)d.nbi * d.nyi + d.na + d.nog + d.mirror_i);
  b += ts * (m * ny + m * d.nbst + m * d.nb + (size_t)d.nb * ny + d.nast + d.na + d.mirror_f);
  return b;
}

void launch_combine3(const DComb3 &d, bool fp64, int grid, int block, cudaStream_t s) {
  size_t smem = combine3_smem(d, fp64);
  int per = (d.nent + block - 1) / block;
  int emax = per <= 2 ? 2 : per <= 4 ? 4 : 8;
  int chunks = (d.nent + block * emax - 1) / (block * emax);
  dim3 g(grid, chunks < 1 ? 1 : chunks);
#define LMFAO_C3(TT, E)                                                                               \
  {                                                                                                   \
    cudaFuncSetAttribute(combine3_kernel<TT, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    combine3_kernel<TT, E><<<g, block, smem, s>>>(d);                                                 \
  }
  if (fp64) {
    if (emax == 2) LMFAO_C3(double, 2) else if (emax == 4) LMFAO_C3(double, 4) else LMFAO_C3(double, 8)
  } else {
    if (emax == 2) LMFAO_C3(float, 2) else if (emax == 4) LMFAO_C3(float, 4) else LMFAO_C3(float, 8)
  }
#undef LMFAO_C3
}

}  // namespace lmfao
