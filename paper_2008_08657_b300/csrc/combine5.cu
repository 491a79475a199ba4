// Two-kernel prefix-block combine (see DComb5 in kernels.cuh).
//
// The outer term of every combine entry factors as psi_t(s) = a_alpha(p) * b_beta(s) over the
// blocks p of m consecutive segments that share the segment-key prefix, so
//     SUM_s psi_t(s) Y_c(s) = SUM_p a_alpha(p) * Z_p[beta][c],   Z_p = B_p^T Y_p
// (the X_A^T C_AB X_B contraction between the prefix-side features a and the block-side
// features b, with the per-segment sums Y of the root pass in the middle).
//
// block_z_kernel: one CTA per block (grid-strided). For each chunk of up to kc segments of the
// block it stages the chunk's per-segment sums with one TMA bulk copy per array (when their
// offsets are 16-byte aligned, else with plain loads), the B-side outer-view columns, the B
// terms, and contracts:
//   * FP32 / FP64: on the CUDA cores from shared memory;
//   * split BF16: on the tensor cores (tcgen05.mma kind::f16, M = 128 rows = Y columns,
//     N = B terms, K = segments), each FP32 operand x split as hi = bf16(x), lo = bf16(x - hi)
//     and Z accumulated as hi*hi + hi*lo + lo*hi in FP32 in tensor memory.
// Integral B terms x integral Y columns are contracted exactly in INT64 on the CUDA cores.
// It also writes the block's A terms and outer cells. Z, A and the cells go to global
// scratch arrays of the plan (L2-resident).
// block_entries_kernel: one thread per (entry, range of blocks): SUM_p a(p) Z_p[b][c] with
// the block's outer cell, flushed into the query outputs (FP64 / INT64 atomics) whenever the
// cell changes.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lmfao {

namespace {

__device__ __forceinline__ int64_t digit5(const DSegment &s, int64_t seg, int i) { return (seg / s.radix[i]) % s.dom[i]; }

template <typename X>
__device__ __forceinline__ bool cmp5(X x, X t, int op) {
  switch (op) {
    case LMFAO_LE: return x <= t;
    case LMFAO_LT: return x < t;
    case LMFAO_GE: return x >= t;
    case LMFAO_GT: return x > t;
    case LMFAO_EQ: return x == t;
    default: return x != t;
  }
}

// Product of a term's segment-digit factors and staged view columns (value and exact integer).
template <typename T>
__device__ __forceinline__ void term5(const DPsi &p, const DSegFac *sf, const int *part, const T *staged,
                                      const DSegment &sg, int64_t seg, T &v, unsigned long long &iv) {
  v = T(1);
  iv = 1ull;
  for (int f = p.f0; f < p.f0 + p.nf; ++f) {
    DSegFac q = sf[f];
    int64_t dg = digit5(sg, seg, q.digit);
    if (q.ind) {
      if (!cmp5<double>((double)dg, (double)q.t, q.op)) { v = T(0); iv = 0; }
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

// ------------------------------------------------------------------ PTX helpers (sm_100 family)
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete; gives up after about a second of
// SM clock (returns false) so that a wait that cannot end does not hold the GPU.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase))
    if (clock64() - t0 > 2000000000ll) return false;
  return true;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand without swizzling: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes; lbo = byte distance between core
// matrices adjacent along K, sbo = between core matrices adjacent along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the sm_100 family; base offset 0; no swizzle
  return d;
}
// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (r, k) of a K-major operand tile with kc columns (no swizzle).
__device__ __forceinline__ uint32_t canon_off(int r, int kq, int kc) {
  return (uint32_t)((((r >> 3) * (kc >> 3)) + kq) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ void split8(const float *x, uint4 &hi, uint4 &lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]), h1 = __float2bfloat16_rn(x[2 * i + 1]);
    __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
    __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
    h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Shared-memory layout of block_z_kernel (byte offsets; the same function sizes the launch).
struct Z5Layout {
  size_t f0, f1, i0, i1, ws, tabs, kmin, bsv, asv, bti, ysf, bt, ahi, alo, bhi, blo, total;
};
__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline Z5Layout z5_layout(const DComb3 &d, int kc, int npad, int ts, int tc) {
  Z5Layout L{};
  size_t o = 0;
  L.f0 = o; o += up16((size_t)kc * d.n0f * ts);  // per-segment float sums are of the pass's type
  L.f1 = o; o += up16((size_t)kc * d.phi1f_seg * 4);
  L.i0 = o; o += up16((size_t)kc * d.n0i * 8);
  L.i1 = o; o += up16((size_t)kc * d.phi1i_seg * 4);
  L.ws = o; o += up16((size_t)kc * 8);
  // B-term tables: descriptors (nb), parts (nbpart), staged columns (nbst)
  L.tabs = o; o += up16((size_t)d.nb * sizeof(DPsi)) + up16((size_t)d.nbpart * 4) + up16((size_t)d.nbst * sizeof(int2));
  L.kmin = o; o += up16((size_t)d.nouter * kc * 8);
  L.bsv = o; o += up16((size_t)kc * d.nbst * ts);
  L.asv = o; o += up16((size_t)d.nast * ts);
  L.bti = o; o += up16((size_t)kc * d.nbi * 8);
  const int ny = d.nyf + d.nyi;
  if (!tc) {
    L.ysf = o; o += up16((size_t)kc * ny * ts);
    L.bt = o; o += up16((size_t)kc * d.nb * ts);
  } else {
    o = (o + 1023) & ~(size_t)1023;
    L.ahi = o; o += (size_t)128 * kc * 2;
    L.alo = o; o += (size_t)128 * kc * 2;
    L.bhi = o; o += (size_t)npad * kc * 2;
    L.blo = o; o += (size_t)npad * kc * 2;
  }
  L.total = o + 1024;  // slack for aligning the dynamic base to 1024 bytes
  return L;
}

template <typename T, int TC>
__global__ void __launch_bounds__(256) block_z_kernel(DComb5 D) {
  const DComb3 &d = D.c;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) unsigned long long bars[2];  // 0: bulk copies, 1: MMA completion
  __shared__ uint32_t tmem_slot;
  __shared__ long long akey[MAXOUT];
  __shared__ int chunk_live, block_live, gave_up;
  const int tid = threadIdx.x, bs = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int kc = D.kc, m = (int)d.m, ny = d.nyf + d.nyi, nb = d.nb, npad = D.npad;
  const Z5Layout L = z5_layout(d, kc, npad, (int)sizeof(T), TC);
  T *f0 = (T *)(smem + L.f0);
  float *f1 = (float *)(smem + L.f1);
  unsigned long long *i0 = (unsigned long long *)(smem + L.i0);
  unsigned int *i1 = (unsigned int *)(smem + L.i1);
  long long *kmin = (long long *)(smem + L.kmin);
  T *bsv = (T *)(smem + L.bsv);
  unsigned long long *bti = (unsigned long long *)(smem + L.bti);
  unsigned long long *ws = (unsigned long long *)(smem + L.ws);
  DPsi *sbterm = (DPsi *)(smem + L.tabs);
  int *sbpart = (int *)(smem + L.tabs + up16((size_t)d.nb * sizeof(DPsi)));
  int2 *sbstage = (int2 *)(smem + L.tabs + up16((size_t)d.nb * sizeof(DPsi)) + up16((size_t)d.nbpart * 4));
  for (int i = tid; i < d.nb; i += bs) sbterm[i] = d.bterm[i];
  for (int i = tid; i < d.nbpart; i += bs) sbpart[i] = d.bpart[i];
  for (int i = tid; i < d.nbst; i += bs) sbstage[i] = d.bstage[i];
  const uint32_t bar_tma = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
  uint32_t ph_tma = 0, ph_mma = 0;
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    fence_mbar_init();
    fence_proxy_async();
    gave_up = 0;
  }
  uint32_t tmem = 0;
  if (TC) {
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                   "r"((uint32_t)D.tmem_cols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // rows of the operands past ny (A) and nb (B) stay zero for the whole launch
    for (int i = tid; i < (128 - ny) * (kc / 8); i += bs) {
      const int r = ny + i % (128 - ny), kq = i / (128 - ny);
      const uint4 z = make_uint4(0, 0, 0, 0);
      *(uint4 *)(smem + L.ahi + canon_off(r, kq, kc)) = z;
      *(uint4 *)(smem + L.alo + canon_off(r, kq, kc)) = z;
    }
    for (int i = tid; i < (npad - nb) * (kc / 8); i += bs) {
      const int r = nb + i % (npad - nb), kq = i / (npad - nb);
      const uint4 z = make_uint4(0, 0, 0, 0);
      *(uint4 *)(smem + L.bhi + canon_off(r, kq, kc)) = z;
      *(uint4 *)(smem + L.blo + canon_off(r, kq, kc)) = z;
    }
    tc_fence_before();
  }
  __syncthreads();
  if (TC) {
    tc_fence_after();
    tmem = tmem_slot;
  }
  const uint32_t idesc = TC ? idesc_bf16(128, npad) : 0u;

  for (int64_t p = blockIdx.x; p < d.nblocks; p += gridDim.x) {
    const int64_t s0 = p * d.m;
    // ---- prefix side: view keys, staged A columns, A terms, outer cells
    if (tid < d.nouter) {
      const DOuter &o = d.outer[tid];
      int64_t k = 0;
      for (int i = 0; i < d.seg.ndig; ++i)
        if (o.dstride[i] && d.seg.radix[i] >= d.m) k += digit5(d.seg, s0, i) * o.dstride[i];
      akey[tid] = k;
    }
    if (tid == 0) block_live = 0;
    __syncthreads();
    {
      T *asv = (T *)(smem + L.asv);
      for (int j = tid; j < d.nast; j += bs) {
        int2 sc = d.astage[j];
        const DOuter &o = d.outer[sc.x];
        asv[j] = (T)__ldg(o.v.v64 + akey[sc.x] * o.v.ncols + sc.y);
      }
      __syncthreads();
      T *ag = (T *)D.a + p * d.na;
      unsigned long long *aig = D.ai + p * d.na;
      for (int a = tid; a < d.na; a += bs) {
        T v;
        unsigned long long iv;
        term5<T>(d.aterm[a], d.segfacs, d.apart, asv, d.seg, s0, v, iv);
        ag[a] = v;
        aig[a] = iv;
      }
      for (int g = tid; g < d.nog; g += bs) {
        long long cell = 0;
        for (int r = d.og_off[g]; r < d.og_off[g + 1] && cell >= 0; ++r) {
          DGroupRef q = d.grefs[r];
          long long code = q.src == 0 ? digit5(d.seg, s0, q.a)
                                      : __ldg(d.outer[q.a].v.codes + akey[q.a] * d.outer[q.a].v.ncodes + q.b);
          if (code < 0) cell = -1;
          else cell += code * q.stride;
        }
        D.cells[p * d.nog + g] = cell;
      }
      __syncthreads();
    }
    // ---- chunks of the block's segments
    for (int k0 = 0; k0 < m; k0 += kc) {
      const int kn = min(kc, m - k0);
      const int64_t sb = s0 + k0;
      // 1. per-segment sums of the chunk into shared memory
      if (D.bulk) {
        if (tid == 0) {
          fence_proxy_async();  // earlier generic reads of these buffers before the async writes
          const uint32_t b0f = (uint32_t)(kn * d.n0f * sizeof(T)), b1f = (uint32_t)(kn * d.phi1f_seg * 4),
                         b0i = (uint32_t)(kn * d.n0i * 8), b1i = (uint32_t)(kn * d.phi1i_seg * 4);
          const uint32_t bws = (uint32_t)(kn * 8);
          mbar_expect_tx(bar_tma, b0f + b1f + b0i + b1i + bws);
          bulk_g2s(smem_u32(ws), d.wseg + sb, bws, bar_tma);
          if (b0f) bulk_g2s(smem_u32(f0), (const T *)d.phi0f + sb * d.n0f, b0f, bar_tma);
          if (b1f) bulk_g2s(smem_u32(f1), d.phi1f + sb * d.phi1f_seg, b1f, bar_tma);
          if (b0i) bulk_g2s(smem_u32(i0), d.phi0i + sb * d.n0i, b0i, bar_tma);
          if (b1i) bulk_g2s(smem_u32(i1), d.phi1i + sb * d.phi1i_seg, b1i, bar_tma);
        }
      } else {
        for (int i = tid; i < kn * d.n0f; i += bs) f0[i] = ((const T *)d.phi0f)[sb * d.n0f + i];
        for (int i = tid; i < kn * (int)d.phi1f_seg; i += bs) f1[i] = d.phi1f[sb * d.phi1f_seg + i];
        for (int i = tid; i < kn * d.n0i; i += bs) i0[i] = d.phi0i[sb * d.n0i + i];
        for (int i = tid; i < kn * (int)d.phi1i_seg; i += bs) i1[i] = d.phi1i[sb * d.phi1i_seg + i];
        for (int i = tid; i < kn; i += bs) ws[i] = d.wseg[sb + i];
      }
      // 2. B-side view columns of the chunk (zero for segments without outer partners)
      if (tid == 0) chunk_live = 0;
      for (int idx = tid; idx < d.nouter * kc; idx += bs) {
        const int o = idx / kc, j = idx - o * kc, jj = k0 + j;
        long long k = 0;
        for (int i = 0; i < d.seg.ndig; ++i)
          if (d.outer[o].dstride[i] && d.seg.radix[i] < d.m) k += ((jj / d.seg.radix[i]) % d.seg.dom[i]) * d.outer[o].dstride[i];
        kmin[idx] = k;
      }
      if (D.bulk) {
        if (!mbar_wait_bounded(bar_tma, ph_tma)) atomicOr(&gave_up, 1);
        ph_tma ^= 1u;
      }
      __syncthreads();
      if (gave_up) break;
      for (int idx = tid; idx < kc * d.nbst; idx += bs) {
        const int s = idx / d.nbst, j = idx - s * d.nbst;
        T v = T(0);
        if (s < kn && ws[s]) {
          chunk_live = 1;
          const int2 sc = sbstage[j];
          const DOuter &o = d.outer[sc.x];
          const int64_t k = akey[sc.x] + kmin[(size_t)sc.x * kc + s];
          v = (T)__ldg(o.v.v64 + k * o.v.ncols + sc.y);
        }
        bsv[idx] = v;
      }
      __syncthreads();
      if (chunk_live && tid == 0) block_live = 1;
      // 3. B terms (integral ones exactly as well)
      // B term b of segment s: product of staged columns (and segment-digit factors, if any)
      auto bterm_at = [&](const DPsi &pt, int s, T &v, unsigned long long &iv) {
        if (pt.nf == 0) {
          v = T(1);
          iv = 1ull;
          const T *row = bsv + (size_t)s * d.nbst;
          for (int i = pt.p0; i < pt.p0 + pt.np; ++i) {
            const T x = row[sbpart[i]];
            v *= x;
            iv *= (unsigned long long)x;
          }
          if (!pt.integral) iv = 0ull;
        } else {
          term5<T>(pt, d.segfacs, sbpart, bsv + (size_t)s * d.nbst, d.seg, sb + s, v, iv);
        }
      };
      if (!TC) {
        T *bt = (T *)(smem + L.bt);
        for (int idx = tid; idx < kc * nb; idx += bs) {
          const int s = idx / nb, b = idx - s * nb;
          T v;
          unsigned long long iv;
          bterm_at(sbterm[b], s, v, iv);
          bt[idx] = v;
          if (b < d.nbi) bti[(size_t)s * d.nbi + b] = iv;
        }
      } else {
        // B operand rows b < nb, 8 segments per item, packed hi / lo BF16
        for (int i = tid; i < nb * (kc / 8); i += bs) {
          const int b = i % nb, kq = i / nb;
          const DPsi pt = sbterm[b];
          float x[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int s = kq * 8 + e;
            T v;
            unsigned long long iv;
            bterm_at(pt, s, v, iv);
            x[e] = s < kn ? (float)v : 0.f;
            if (b < d.nbi) bti[(size_t)s * d.nbi + b] = iv;
          }
          uint4 hi, lo;
          split8(x, hi, lo);
          *(uint4 *)(smem + L.bhi + canon_off(b, kq, kc)) = hi;
          *(uint4 *)(smem + L.blo + canon_off(b, kq, kc)) = lo;
        }
      }
      // 4. the Y operand
      auto yval = [&](int s, int c) -> T {
        if (c < d.n0f) return (T)f0[s * d.n0f + c];
        if (c < d.nyf) return (T)f1[s * (int)d.phi1f_seg + (c - d.n0f)];
        const int ci = c - d.nyf;
        return ci < d.n0i ? (T)i0[s * d.n0i + ci] : (T)i1[s * (int)d.phi1i_seg + (ci - d.n0i)];
      };
      if (!TC) {
        T *ysf = (T *)(smem + L.ysf);
        for (int idx = tid; idx < kc * ny; idx += bs) {
          const int s = idx / ny, c = idx - s * ny;
          ysf[idx] = s < kn ? yval(s, c) : T(0);
        }
      } else {
        for (int i = tid; i < ny * (kc / 8); i += bs) {
          const int c = i % ny, kq = i / ny;
          float x[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int s = kq * 8 + e;
            x[e] = s < kn ? (float)yval(s, c) : 0.f;
          }
          uint4 hi, lo;
          split8(x, hi, lo);
          *(uint4 *)(smem + L.ahi + canon_off(c, kq, kc)) = hi;
          *(uint4 *)(smem + L.alo + canon_off(c, kq, kc)) = lo;
        }
        fence_proxy_async();  // generic-proxy writes of the operands -> visible to the MMA
      }
      __syncthreads();
      // 5. contraction of the chunk
      if (TC) {
        if (tid == 0) {
          tc_fence_after();
          const uint32_t sbo = (uint32_t)kc * 16u;
          const uint32_t ah = smem_u32(smem + L.ahi), al = smem_u32(smem + L.alo);
          const uint32_t bh = smem_u32(smem + L.bhi), bl = smem_u32(smem + L.blo);
          for (int j = 0; j < kc / 16; ++j) {
            const uint32_t off = (uint32_t)j * 256u;
            const uint32_t acc0 = (k0 > 0 || j > 0) ? 1u : 0u;
            // small terms first: lo*hi and hi*lo, then hi*hi
            umma_bf16(tmem, smem_desc(al + off, 128, sbo), smem_desc(bh + off, 128, sbo), idesc, acc0);
            umma_bf16(tmem, smem_desc(ah + off, 128, sbo), smem_desc(bl + off, 128, sbo), idesc, 1u);
            umma_bf16(tmem, smem_desc(ah + off, 128, sbo), smem_desc(bh + off, 128, sbo), idesc, 1u);
          }
          umma_commit(bar_mma);
        }
      } else {
        const T *bt = (const T *)(smem + L.bt);
        const T *ysf = (const T *)(smem + L.ysf);
        const int nq = (ny + 3) >> 2;
        T *zg = (T *)D.z + p * (int64_t)nb * ny;
        for (int o = tid; o < nb * nq; o += bs) {
          const int b = o / nq, c0 = 4 * (o - b * nq);
          T z0 = T(0), z1 = T(0), z2 = T(0), z3 = T(0);
          if (c0 + 3 < ny) {
            for (int s = 0; s < kn; ++s) {
              const T bv = bt[(size_t)s * nb + b];
              const T *y = ysf + (size_t)s * ny + c0;
              z0 += bv * y[0];
              z1 += bv * y[1];
              z2 += bv * y[2];
              z3 += bv * y[3];
            }
          } else {
            for (int s = 0; s < kn; ++s) {
              const T bv = bt[(size_t)s * nb + b];
              const T *y = ysf + (size_t)s * ny + c0;
              z0 += bv * y[0];
              if (c0 + 1 < ny) z1 += bv * y[1];
              if (c0 + 2 < ny) z2 += bv * y[2];
            }
          }
          T *zo = zg + (size_t)b * ny + c0;
          if (k0 == 0) {
            zo[0] = z0;
            if (c0 + 1 < ny) zo[1] = z1;
            if (c0 + 2 < ny) zo[2] = z2;
            if (c0 + 3 < ny) zo[3] = z3;
          } else {
            zo[0] += z0;
            if (c0 + 1 < ny) zo[1] += z1;
            if (c0 + 2 < ny) zo[2] += z2;
            if (c0 + 3 < ny) zo[3] += z3;
          }
        }
      }
      // exact integral part: integral B terms x integral Y columns
      {
        unsigned long long *zig = D.zi + p * (int64_t)d.nbi * d.nyi;
        for (int o = tid; o < d.nbi * d.nyi; o += bs) {
          const int b = o / d.nyi, c = o - b * d.nyi;
          unsigned long long z = 0;
          for (int s = 0; s < kn; ++s) {
            const unsigned long long y =
                c < d.n0i ? i0[s * d.n0i + c] : (unsigned long long)i1[s * (int)d.phi1i_seg + (c - d.n0i)];
            z += bti[(size_t)s * d.nbi + b] * y;
          }
          zig[o] = k0 == 0 ? z : zig[o] + z;
        }
      }
      if (TC) {
        // the next chunk rewrites the operands: wait for this chunk's MMAs
        if (!mbar_wait_bounded(bar_mma, ph_mma)) atomicOr(&gave_up, 1);
        ph_mma ^= 1u;
        tc_fence_after();
      }
      __syncthreads();
      if (gave_up) break;
    }
    if (gave_up) break;
    if (TC) {
      // Z from tensor memory: lane c of warp w % 4 holds row c = 32 (w % 4) + lane; the two
      // warp groups take alternate 8-column groups of the npad B terms
      const int c = 32 * (warp & 3) + lane;
      T *zg = (T *)D.z + p * (int64_t)nb * ny;
      for (int g = warp >> 2; g < npad / 8; g += bs / 128) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(8 * g), v);
        if (c < ny) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (8 * g + e < nb) zg[(size_t)(8 * g + e) * ny + c] = (T)v[e];
        }
      }
      tc_fence_before();
    }
    if (tid == 0) D.live[p] = block_live;
    __syncthreads();
  }
  if (TC) {
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)D.tmem_cols)
                   : "memory");
  }
  if (gave_up && tid == 0) atomicOr(D.err, 8);
}

// ------------------------------------------------------------------ dense-B contraction
// When every B term is one column of an outer view (or the constant 1) with no segment-digit
// factor, a chunk's B operand is read straight from the view rows. block_zd_kernel keeps the
// block's Z_p in registers, 4 x 4 tiles (4 B terms x 4 Y columns, read from shared memory with
// one 16-byte load each per segment) of which each thread owns KT, accumulated over the block's
// chunks and written once. The chunk's operands are staged by warps over rows and lanes over
// columns (coalesced, no index division); the exact integral part is spread over all threads
// and summed in shared memory. The small shared footprint leaves several CTAs per SM, so one
// CTA's loads overlap another's multiply-adds.
constexpr int kZq = 4;  // tile edge
constexpr int kZl = 4;  // operand columns per lane in staging (Y and B of at most 128 columns)

struct ZdLayout {
  size_t ysf, bt, yi0, yi1, bti, lv, kmin, asv, zacc, bsrc, total;
};
__host__ __device__ inline ZdLayout zd_layout(const DComb3 &d, int kc, int ts) {
  const int ny = d.nyf + d.nyi;
  const size_t nyp = (size_t)(ny + kZq - 1) / kZq * kZq, nbp = (size_t)(d.nb + kZq - 1) / kZq * kZq;
  ZdLayout L{};
  size_t o = 0;
  L.ysf = o; o += up16((size_t)kc * nyp * ts);
  L.bt = o; o += up16((size_t)kc * nbp * ts);
  L.yi0 = o; o += up16((size_t)kc * d.n0i * 8);
  L.yi1 = o; o += up16((size_t)kc * (d.nyi - d.n0i) * 4);
  L.bti = o; o += up16((size_t)kc * d.nbi * 8);
  L.lv = o; o += up16((size_t)kc * 4);
  L.kmin = o; o += up16((size_t)d.nouter * kc * 8);
  L.asv = o; o += up16((size_t)d.nast * ts);
  L.zacc = o; o += up16((size_t)d.nbi * d.nyi * 8);
  L.bsrc = o; o += up16((size_t)d.nb * 8);
  L.total = o;
  return L;
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  __device__ static void load(const float *p, float (&v)[4]) {
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  }
};
template <>
struct Vec4<double> {
  __device__ static void load(const double *p, double (&v)[4]) {
    const double2 x = reinterpret_cast<const double2 *>(p)[0], y = reinterpret_cast<const double2 *>(p)[1];
    v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
  }
};

template <typename T, int KT>
__global__ void __launch_bounds__(256) block_zd_kernel(DComb5 D) {
  const DComb3 &d = D.c;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long akey[MAXOUT];
  __shared__ int block_live;
  const int tid = threadIdx.x, bs = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = bs >> 5;
  const int kc = D.kc, m = (int)d.m, ny = d.nyf + d.nyi, nb = d.nb, nyi1 = d.nyi - d.n0i;
  const int nyp = (ny + kZq - 1) / kZq * kZq, nbp = (nb + kZq - 1) / kZq * kZq;
  const int nct = nyp / kZq, ntile = (nbp / kZq) * nct, nzi = d.nbi * d.nyi;
  const ZdLayout L = zd_layout(d, kc, (int)sizeof(T));
  T *ysf = (T *)(smem + L.ysf);
  T *bt = (T *)(smem + L.bt);
  unsigned long long *yi0 = (unsigned long long *)(smem + L.yi0);
  unsigned int *yi1 = (unsigned int *)(smem + L.yi1);
  unsigned long long *bti = (unsigned long long *)(smem + L.bti);
  int *lv = (int *)(smem + L.lv);
  long long *kmin = (long long *)(smem + L.kmin);
  T *asv = (T *)(smem + L.asv);
  unsigned long long *zacc = (unsigned long long *)(smem + L.zacc);
  // the B terms' sources, read by every staged row
  int2 *sbsrc = (int2 *)(smem + L.bsrc);
  for (int b = tid; b < nb; b += bs) sbsrc[b] = D.bsrc[b];
  for (int64_t p = blockIdx.x; p < d.nblocks; p += gridDim.x) {
    const int64_t s0 = p * d.m;
    // ---- prefix side (as in block_z_kernel): view keys, A terms, outer cells
    if (tid < d.nouter) {
      const DOuter &o = d.outer[tid];
      int64_t k = 0;
      for (int i = 0; i < d.seg.ndig; ++i)
        if (o.dstride[i] && d.seg.radix[i] >= d.m) k += digit5(d.seg, s0, i) * o.dstride[i];
      akey[tid] = k;
    }
    if (tid == 0) block_live = 0;
    for (int i = tid; i < nzi; i += bs) zacc[i] = 0ull;
    __syncthreads();
    for (int j = tid; j < d.nast; j += bs) {
      const int2 sc = d.astage[j];
      const DOuter &o = d.outer[sc.x];
      asv[j] = (T)__ldg(o.v.v64 + akey[sc.x] * o.v.ncols + sc.y);
    }
    __syncthreads();
    {
      T *ag = (T *)D.a + p * d.na;
      unsigned long long *aig = D.ai + p * d.na;
      for (int a = tid; a < d.na; a += bs) {
        T v;
        unsigned long long iv;
        term5<T>(d.aterm[a], d.segfacs, d.apart, asv, d.seg, s0, v, iv);
        ag[a] = v;
        aig[a] = iv;
      }
      for (int g = tid; g < d.nog; g += bs) {
        long long cell = 0;
        for (int r = d.og_off[g]; r < d.og_off[g + 1] && cell >= 0; ++r) {
          const DGroupRef q = d.grefs[r];
          const long long code = q.src == 0 ? digit5(d.seg, s0, q.a)
                                            : __ldg(d.outer[q.a].v.codes + akey[q.a] * d.outer[q.a].v.ncodes + q.b);
          if (code < 0) cell = -1;
          else cell += code * q.stride;
        }
        D.cells[p * d.nog + g] = cell;
      }
    }
    T acc[KT][kZq * kZq];
#pragma unroll
    for (int t = 0; t < KT; ++t)
#pragma unroll
      for (int i = 0; i < kZq * kZq; ++i) acc[t][i] = T(0);
    for (int k0 = 0; k0 < m; k0 += kc) {
      const int kn = min(kc, m - k0);
      const int64_t sb = s0 + k0;
      // 1. liveness and the minor-digit part of each B-side view key
      for (int i = tid; i < kn; i += bs) lv[i] = d.wseg[sb + i] != 0ull;
      for (int o = 0; o < d.nouter; ++o)
        for (int j = tid; j < kn; j += bs) {
          const int jj = k0 + j;
          long long k = 0;
          for (int i = 0; i < d.seg.ndig; ++i)
            if (d.outer[o].dstride[i] && d.seg.radix[i] < d.m)
              k += ((jj / d.seg.radix[i]) % d.seg.dom[i]) * d.outer[o].dstride[i];
          kmin[o * kc + j] = k;
        }
      __syncthreads();
      // 2. operands, one warp per segment row: Y (integral columns also exactly) and B (zero
      // on segments without outer partners; integral B terms also exactly)
      for (int s = warp; s < kn; s += nwarp) {
        const int64_t g = sb + s;
        const T *f0 = (const T *)d.phi0f + g * d.n0f;
        const float *f1 = d.phi1f + g * d.phi1f_seg;
        const unsigned long long *i0 = d.phi0i + g * d.n0i;
        const unsigned int *i1 = d.phi1i + g * d.phi1i_seg;
#pragma unroll
        for (int i = 0; i < kZl; ++i) {
          const int c = lane + 32 * i;
          if (c >= nyp) break;
          T v = T(0);
          // the Y array of column c: 0 float sums, 1 float cells, 2 integral sums, 3 integral cells
          switch (c >= ny ? -1 : c < d.n0f ? 0 : c < d.nyf ? 1 : c < d.nyf + d.n0i ? 2 : 3) {
            case 0: v = f0[c]; break;
            case 1: v = (T)f1[c - d.n0f]; break;
            case 2: {
              const unsigned long long y = i0[c - d.nyf];
              yi0[s * d.n0i + (c - d.nyf)] = y;
              v = (T)y;
              break;
            }
            case 3: {
              const unsigned int y = i1[c - d.nyf - d.n0i];
              yi1[s * nyi1 + (c - d.nyf - d.n0i)] = y;
              v = (T)y;
              break;
            }
            default: break;
          }
          ysf[s * nyp + c] = v;
        }
        const bool live = lv[s] != 0;
#pragma unroll
        for (int i = 0; i < kZl; ++i) {
          const int b = lane + 32 * i;
          if (b >= nbp) break;
          T v = T(0);
          unsigned long long iv = 0ull;
          if (b < nb && live) {
            const int2 src = sbsrc[b];
            if (src.x < 0) {
              v = T(1);
              iv = 1ull;
            } else {
              const DOuter &o = d.outer[src.x];
              const double x = __ldg(o.v.v64 + (akey[src.x] + kmin[src.x * kc + s]) * o.v.ncols + src.y);
              v = (T)x;
              iv = (unsigned long long)x;
            }
          }
          bt[s * nbp + b] = v;
          if (b < d.nbi) bti[s * d.nbi + b] = iv;
        }
        if (lane == 0 && live) block_live = 1;
      }
      __syncthreads();
      // 3. the contraction into the register tiles
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int tile = tid + t * bs;
        if (tile < ntile) {
          const int b0 = (tile / nct) * kZq, c0 = (tile - (tile / nct) * nct) * kZq;
          const T *br = bt + b0, *yr = ysf + c0;
          for (int s = 0; s < kn; ++s, br += nbp, yr += nyp) {
            T bv[4], yv[4];
            Vec4<T>::load(br, bv);
            Vec4<T>::load(yr, yv);
#pragma unroll
            for (int i = 0; i < kZq; ++i)
#pragma unroll
              for (int j = 0; j < kZq; ++j) acc[t][i * kZq + j] += bv[i] * yv[j];
          }
        }
      }
      // 4. integral B terms x integral Y columns, exactly: (output, 8-segment run) per thread
      for (int w = tid; w < nzi * ((kn + 7) >> 3); w += bs) {
        const int o = w % nzi, s1 = (w / nzi) * 8, s2 = min(kn, s1 + 8);
        const int b = o / d.nyi, c = o - b * d.nyi;
        unsigned long long z = 0;
        for (int s = s1; s < s2; ++s)
          z += bti[s * d.nbi + b] * (c < d.n0i ? yi0[s * d.n0i + c] : (unsigned long long)yi1[s * nyi1 + (c - d.n0i)]);
        if (z) atomicAdd(zacc + o, z);
      }
      __syncthreads();
    }
    T *zg = (T *)D.z + p * (int64_t)nb * ny;
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int tile = tid + t * bs;
      if (tile < ntile) {
        const int b0 = (tile / nct) * kZq, c0 = (tile - (tile / nct) * nct) * kZq;
#pragma unroll
        for (int i = 0; i < kZq; ++i)
#pragma unroll
          for (int j = 0; j < kZq; ++j)
            if (b0 + i < nb && c0 + j < ny) zg[(size_t)(b0 + i) * ny + c0 + j] = acc[t][i * kZq + j];
      }
    }
    unsigned long long *zig = D.zi + p * (int64_t)nzi;
    for (int i = tid; i < nzi; i += bs) zig[i] = zacc[i];
    if (tid == 0) D.live[p] = block_live;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ pipelined dense contraction
// block_zp_kernel: block_zd_kernel with the operand reads made asynchronous. Every thread
// issues cp.async copies (4 or 8 bytes each, so no alignment beyond the element's is needed)
// of the next chunk's per-segment sums, segment weights and B-side view values into the other
// of two raw stages while the current chunk is converted and contracted; a CTA's chunks run in
// one sequence across its blocks, so the next block's first chunk is in flight during the last
// chunk of the current one.
struct ZpLayout {
  size_t rf0, rf1, ri0, ri1, rws, rb, stage, ysf, bt, bti, lv, asv, zacc, bsrc, total;  // raw stage st at st * stage
};
__host__ __device__ inline ZpLayout zp_layout(const DComb3 &d, int kc, int ts) {
  const int ny = d.nyf + d.nyi;
  const size_t nyp = (size_t)(ny + kZq - 1) / kZq * kZq, nbp = (size_t)(d.nb + kZq - 1) / kZq * kZq;
  ZpLayout L{};
  size_t o = 0;  // offsets inside one raw stage
  L.rf0 = o; o += up16((size_t)kc * d.n0f * ts);
  L.rf1 = o; o += up16((size_t)kc * d.phi1f_seg * 4);
  L.ri0 = o; o += up16((size_t)kc * d.n0i * 8);
  L.ri1 = o; o += up16((size_t)kc * d.phi1i_seg * 4);
  L.rws = o; o += up16((size_t)kc * 8);
  L.rb = o; o += up16((size_t)kc * d.nb * 8);
  L.stage = o;
  o *= 2;
  L.ysf = o; o += up16((size_t)kc * nyp * ts);
  L.bt = o; o += up16((size_t)kc * nbp * ts);
  L.bti = o; o += up16((size_t)kc * d.nbi * 8);
  L.lv = o; o += up16((size_t)kc * 4);
  L.asv = o; o += up16((size_t)d.nast * ts);
  L.zacc = o; o += up16((size_t)d.nbi * d.nyi * 8);
  L.bsrc = o; o += up16((size_t)d.nb * 8);
  L.total = o;
  return L;
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

template <typename T, int KT>
__global__ void __launch_bounds__(256, KT == 1 && sizeof(T) == 4 ? 4 : 2) block_zp_kernel(DComb5 D) {
  const DComb3 &d = D.c;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long akey[MAXOUT];
  __shared__ int block_live;
  const int tid = threadIdx.x, bs = blockDim.x;
  const int kc = D.kc, m = (int)d.m, ny = d.nyf + d.nyi, nb = d.nb;
  const int nyp = (ny + kZq - 1) / kZq * kZq, nbp = (nb + kZq - 1) / kZq * kZq;
  const int nct = nyp / kZq, ntile = (nbp / kZq) * nct, nzi = d.nbi * d.nyi;
  const int ts = (int)sizeof(T);
  const ZpLayout L = zp_layout(d, kc, ts);
  T *ysf = (T *)(smem + L.ysf);
  T *bt = (T *)(smem + L.bt);
  unsigned long long *bti = (unsigned long long *)(smem + L.bti);
  int *lv = (int *)(smem + L.lv);
  T *asv = (T *)(smem + L.asv);
  unsigned long long *zacc = (unsigned long long *)(smem + L.zacc);
  int2 *sbsrc = (int2 *)(smem + L.bsrc);
  for (int b = tid; b < nb; b += bs) sbsrc[b] = D.bsrc[b];
  const DOuter &ob = d.outer[D.bout];
  const int nchunk = (m + kc - 1) / kc;
  const int64_t nitems = ((d.nblocks - blockIdx.x + gridDim.x - 1) / gridDim.x) * nchunk;
  __syncthreads();  // sbsrc
  // row of outer view bout at the prefix digits of block p
  auto brow0 = [&](int64_t p) {
    int64_t k = 0;
    const int64_t s0 = p * d.m;
    for (int i = 0; i < d.seg.ndig; ++i)
      if (ob.dstride[i] && d.seg.radix[i] >= d.m) k += digit5(d.seg, s0, i) * ob.dstride[i];
    return k;
  };
  // copies of item it (block, chunk) into raw stage st
  auto issue = [&](int64_t it, int st) {
    const int64_t p = blockIdx.x + (it / nchunk) * gridDim.x;
    const int k0 = (int)(it % nchunk) * kc, kn = min(kc, m - k0);
    const int64_t sb = p * d.m + k0;
    unsigned char *raw = smem + (st ? L.stage : 0);
    for (int i = tid; i < kn * d.n0f; i += bs)
      if (ts == 8) cp_async8(raw + L.rf0 + (size_t)i * 8, (const T *)d.phi0f + sb * d.n0f + i);
      else cp_async4(raw + L.rf0 + (size_t)i * 4, (const T *)d.phi0f + sb * d.n0f + i);
    for (int i = tid; i < kn * (int)d.phi1f_seg; i += bs) cp_async4(raw + L.rf1 + (size_t)i * 4, d.phi1f + sb * d.phi1f_seg + i);
    for (int i = tid; i < kn * d.n0i; i += bs) cp_async8(raw + L.ri0 + (size_t)i * 8, d.phi0i + sb * d.n0i + i);
    for (int i = tid; i < kn * (int)d.phi1i_seg; i += bs) cp_async4(raw + L.ri1 + (size_t)i * 4, d.phi1i + sb * d.phi1i_seg + i);
    for (int i = tid; i < kn; i += bs) cp_async8(raw + L.rws + (size_t)i * 8, d.wseg + sb + i);
    const double *vrow = ob.v.v64 + (brow0(p) + (int64_t)k0 * D.bstride) * ob.v.ncols;
    const int64_t rstride = D.bstride * ob.v.ncols;
    for (int i = tid; i < kn * nb; i += bs) {
      const int s = i / nb, b = i - s * nb;
      const int2 src = sbsrc[b];
      if (src.x >= 0) cp_async8(raw + L.rb + (size_t)i * 8, vrow + (int64_t)s * rstride + src.y);
    }
  };
  if (nitems > 0) issue(0, 0);
  cp_async_commit();
  T acc[KT][kZq * kZq];
  for (int64_t it = 0; it < nitems; ++it) {
    const int st = (int)(it & 1);
    const int64_t p = blockIdx.x + (it / nchunk) * gridDim.x;
    const int k0 = (int)(it % nchunk) * kc, kn = min(kc, m - k0);
    const int64_t s0 = p * d.m;
    if (k0 == 0) {
      // ---- prefix side (as in block_z_kernel): view keys, A terms, outer cells
      if (tid < d.nouter) {
        const DOuter &o = d.outer[tid];
        int64_t k = 0;
        for (int i = 0; i < d.seg.ndig; ++i)
          if (o.dstride[i] && d.seg.radix[i] >= d.m) k += digit5(d.seg, s0, i) * o.dstride[i];
        akey[tid] = k;
      }
      if (tid == 0) block_live = 0;
      for (int i = tid; i < nzi; i += bs) zacc[i] = 0ull;
      __syncthreads();
      for (int j = tid; j < d.nast; j += bs) {
        const int2 sc = d.astage[j];
        const DOuter &o = d.outer[sc.x];
        asv[j] = (T)__ldg(o.v.v64 + akey[sc.x] * o.v.ncols + sc.y);
      }
      __syncthreads();
      T *ag = (T *)D.a + p * d.na;
      unsigned long long *aig = D.ai + p * d.na;
      for (int a = tid; a < d.na; a += bs) {
        T v;
        unsigned long long iv;
        term5<T>(d.aterm[a], d.segfacs, d.apart, asv, d.seg, s0, v, iv);
        ag[a] = v;
        aig[a] = iv;
      }
      for (int g = tid; g < d.nog; g += bs) {
        long long cell = 0;
        for (int r = d.og_off[g]; r < d.og_off[g + 1] && cell >= 0; ++r) {
          const DGroupRef q = d.grefs[r];
          const long long code = q.src == 0 ? digit5(d.seg, s0, q.a)
                                            : __ldg(d.outer[q.a].v.codes + akey[q.a] * d.outer[q.a].v.ncodes + q.b);
          if (code < 0) cell = -1;
          else cell += code * q.stride;
        }
        D.cells[p * d.nog + g] = cell;
      }
#pragma unroll
      for (int t = 0; t < KT; ++t)
#pragma unroll
        for (int i = 0; i < kZq * kZq; ++i) acc[t][i] = T(0);
    }
    // the next item's copies go to the other stage (free: its conversion ended before the
    // barrier that closed the previous item)
    if (it + 1 < nitems) issue(it + 1, st ^ 1);
    cp_async_commit();
    cp_async_wait1();  // this item's copies
    __syncthreads();
    // convert the raw stage: Y (FP32 / FP64, integral columns as numbers), B (zero without
    // outer partners), integral B terms exactly
    const unsigned char *raw = smem + (st ? L.stage : 0);
    const T *rf0 = (const T *)(raw + L.rf0);
    const float *rf1 = (const float *)(raw + L.rf1);
    const unsigned long long *ri0 = (const unsigned long long *)(raw + L.ri0);
    const unsigned int *ri1 = (const unsigned int *)(raw + L.ri1);
    const unsigned long long *rws = (const unsigned long long *)(raw + L.rws);
    const double *rb = (const double *)(raw + L.rb);
    for (int i = tid; i < kn; i += bs) {
      lv[i] = rws[i] != 0ull;
      if (rws[i] != 0ull) block_live = 1;
    }
    for (int i = tid; i < kn * nyp; i += bs) {
      const int s = i / nyp, c = i - s * nyp;
      T v = T(0);
      if (c < d.n0f) v = rf0[s * d.n0f + c];
      else if (c < d.nyf) v = (T)rf1[s * (int)d.phi1f_seg + (c - d.n0f)];
      else if (c < d.nyf + d.n0i) v = (T)ri0[s * d.n0i + (c - d.nyf)];
      else if (c < ny) v = (T)ri1[s * (int)d.phi1i_seg + (c - d.nyf - d.n0i)];
      ysf[i] = v;
    }
    for (int i = tid; i < kn * nbp; i += bs) {
      const int s = i / nbp, b = i - s * nbp;
      T v = T(0);
      unsigned long long iv = 0ull;
      if (b < nb && rws[s] != 0ull) {
        if (sbsrc[b].x < 0) {
          v = T(1);
          iv = 1ull;
        } else {
          const double x = rb[s * nb + b];
          v = (T)x;
          iv = (unsigned long long)x;
        }
      }
      bt[i] = v;
      if (b < d.nbi) bti[s * d.nbi + b] = iv;
    }
    __syncthreads();
    // contraction into the register tiles
#pragma unroll
    for (int t = 0; t < KT; ++t) {
      const int tile = tid + t * bs;
      if (tile < ntile) {
        const int b0 = (tile / nct) * kZq, c0 = (tile - (tile / nct) * nct) * kZq;
        const T *br = bt + b0, *yr = ysf + c0;
        for (int s = 0; s < kn; ++s, br += nbp, yr += nyp) {
          T bv[4], yv[4];
          Vec4<T>::load(br, bv);
          Vec4<T>::load(yr, yv);
#pragma unroll
          for (int i = 0; i < kZq; ++i)
#pragma unroll
            for (int j = 0; j < kZq; ++j) acc[t][i * kZq + j] += bv[i] * yv[j];
        }
      }
    }
    // integral B terms x integral Y columns, exactly: (output, 8-segment run) per thread
    for (int w = tid; w < nzi * ((kn + 7) >> 3); w += bs) {
      const int o = w % nzi, s1 = (w / nzi) * 8, s2 = min(kn, s1 + 8);
      const int b = o / d.nyi, c = o - b * d.nyi;
      unsigned long long z = 0;
      for (int s = s1; s < s2; ++s)
        z += bti[s * d.nbi + b] * (c < d.n0i ? ri0[s * d.n0i + c] : (unsigned long long)ri1[s * (int)d.phi1i_seg + (c - d.n0i)]);
      if (z) atomicAdd(zacc + o, z);
    }
    if (k0 + kn >= m) {  // the block's last chunk
      __syncthreads();
      T *zg = (T *)D.z + p * (int64_t)nb * ny;
#pragma unroll
      for (int t = 0; t < KT; ++t) {
        const int tile = tid + t * bs;
        if (tile < ntile) {
          const int b0 = (tile / nct) * kZq, c0 = (tile - (tile / nct) * nct) * kZq;
#pragma unroll
          for (int i = 0; i < kZq; ++i)
#pragma unroll
            for (int j = 0; j < kZq; ++j)
              if (b0 + i < nb && c0 + j < ny) zg[(size_t)(b0 + i) * ny + c0 + j] = acc[t][i * kZq + j];
        }
      }
      unsigned long long *zig = D.zi + p * (int64_t)nzi;
      for (int i = tid; i < nzi; i += bs) zig[i] = zacc[i];
      if (tid == 0) D.live[p] = block_live;
    }
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// SUM_p a(p) Z_p[b][c] per entry, one thread per (entry, range of blocks).
template <typename T>
__global__ void __launch_bounds__(256) block_entries_kernel(DComb5 D) {
  const DComb3 &d = D.c;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.nent) return;
  const int64_t per = (d.nblocks + gridDim.y - 1) / gridDim.y;
  const int64_t p0 = (int64_t)blockIdx.y * per, p1 = min(d.nblocks, p0 + per);
  if (p0 >= p1) return;
  const DEntry3 en = d.ent[e];
  const int ny = d.nyf + d.nyi;
  const int64_t zs = (int64_t)d.nb * ny, zis = (int64_t)d.nbi * d.nyi;
  const int64_t zoff = (int64_t)en.b * ny + (en.yint ? d.nyf + en.c : en.c);
  const int64_t zioff = (int64_t)en.b * d.nyi + en.c;
  long long cur = -1;
  double accf = 0.0;
  unsigned long long acci = 0ull;
  auto flush = [&]() {
    if (cur < 0) return;
    const long long rel = (cur + en.icell) * en.cellmul;
    if (en.integral) {
      if (acci) atomicAdd(d.icnt + en.out + rel, acci);
    } else if (accf != 0.0) {
      atomicAdd(d.fsum + en.out + rel, accf);
    }
    accf = 0.0;
    acci = 0ull;
  };
  const T *A = (const T *)D.a;
  const T *Z = (const T *)D.z;
  for (int64_t p = p0; p < p1; ++p) {
    if (!D.live[p]) continue;
    const long long cell = D.cells[p * d.nog + en.og];
    if (cell < 0) continue;
    if (cell != cur) {
      flush();
      cur = cell;
    }
    if (en.integral) acci += D.ai[p * d.na + en.a] * D.zi[p * zis + zioff];
    else accf += (double)(A[p * d.na + en.a] * Z[p * zs + zoff]);
  }
  flush();
}

}  // namespace

size_t combine5_smem(const DComb5 &D, bool fp64) {
  if (D.pipe) return zp_layout(D.c, D.kc, fp64 ? 8 : 4).total;
  if (D.dense) return zd_layout(D.c, D.kc, fp64 ? 8 : 4).total;
  return z5_layout(D.c, D.kc, D.npad, fp64 ? 8 : 4, D.tc).total;
}

static int zd_ntile(const DComb3 &d) {
  const int ny = d.nyf + d.nyi;
  return ((d.nb + kZq - 1) / kZq) * ((ny + kZq - 1) / kZq);
}

bool combine5_dense_fits(const DComb3 &d) {
  const int ny = d.nyf + d.nyi;
  return zd_ntile(d) <= 2 * 256 && (ny + kZq - 1) / kZq * kZq <= 32 * kZl && (d.nb + kZq - 1) / kZq * kZq <= 32 * kZl;
}

template <typename T, int KT>
static void launch_zd(const DComb5 &D, size_t smem, cudaStream_t s) {
  cudaFuncSetAttribute(block_zd_kernel<T, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1, dev = 0, nsm = 148;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_zd_kernel<T, KT>, 256, smem);
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(D.c.nblocks, (int64_t)nsm * std::max(1, per_sm)));
  block_zd_kernel<T, KT><<<grid, 256, smem, s>>>(D);
}

template <typename T, int KT>
static void launch_zp(const DComb5 &D, size_t smem, cudaStream_t s) {
  cudaFuncSetAttribute(block_zp_kernel<T, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1, dev = 0, nsm = 148;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, block_zp_kernel<T, KT>, 256, smem);
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(D.c.nblocks, (int64_t)nsm * std::max(1, per_sm)));
  block_zp_kernel<T, KT><<<grid, 256, smem, s>>>(D);
}

void launch_combine5_z(const DComb5 &D, bool fp64, cudaStream_t s) {
  const size_t smem = combine5_smem(D, fp64);
  if (D.pipe) {
    const bool one = zd_ntile(D.c) <= 256;
    if (fp64) one ? launch_zp<double, 1>(D, smem, s) : launch_zp<double, 2>(D, smem, s);
    else one ? launch_zp<float, 1>(D, smem, s) : launch_zp<float, 2>(D, smem, s);
    return;
  }
  if (D.dense) {
    const bool one = zd_ntile(D.c) <= 256;  // one tile per thread
    if (fp64) one ? launch_zd<double, 1>(D, smem, s) : launch_zd<double, 2>(D, smem, s);
    else one ? launch_zd<float, 1>(D, smem, s) : launch_zd<float, 2>(D, smem, s);
    return;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(D.c.nblocks, (int64_t)D.grid));
#define LMFAO_Z5(TT, TCV)                                                                                    \
  {                                                                                                          \
    cudaFuncSetAttribute(block_z_kernel<TT, TCV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);   \
    block_z_kernel<TT, TCV><<<grid, 256, smem, s>>>(D);                                                      \
  }
  if (fp64) LMFAO_Z5(double, 0)
  else if (D.tc) LMFAO_Z5(float, 1)
  else LMFAO_Z5(float, 0)
#undef LMFAO_Z5
}

void launch_combine5_entries(const DComb5 &D, bool fp64, cudaStream_t s) {
  if (D.c.nent == 0) return;
  dim3 g((unsigned)((D.c.nent + 255) / 256), (unsigned)std::max(1, D.eranges));
  if (fp64) block_entries_kernel<double><<<g, 256, 0, s>>>(D);
  else block_entries_kernel<float><<<g, 256, 0, s>>>(D);
}

}  // namespace lmfao
