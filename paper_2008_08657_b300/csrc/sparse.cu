// COUNT GROUP BY over the natural join with the groups kept in hash tables (the group-bys of
// Rk-means, Section 3: SUM(1) GROUP BY X_j over the values of one attribute, and SUM(1) GROUP
// BY C_1, ..., C_n over the cells of a grid of cluster intervals). The key spaces of these
// group-bys are far too large for dense result cells, so:
//
//  * every group attribute has a code (a categorical or key value, a bucket index, or the
//    32-bit pattern of an FP32 value) and the group key of a joined tuple is the mixed-radix
//    number of its codes (at most 62 bits);
//  * each non-root relation, in post-order of the join tree, gets a partial view keyed by its
//    join key toward the parent: the multiplicity of the key in its subtree and the part of
//    the group key that the attributes of its subtree contribute (they must be determined by
//    the join key, as the views of the engine require);
//  * the root pass forms each tuple's key from its own attributes and its children's partial
//    views and counts it in a per-CTA open-addressing table in shared memory; a key that does
//    not find a slot there within a few probes goes to the global table in HBM (linear probing
//    over 2^k slots of 64-bit keys and counts), and each CTA's table is flushed into the global
//    table at the end.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace lmfao {

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kCtaSlots = 2048;  // per-CTA table (16 KB of keys + 16 KB of counts)
constexpr int kCtaProbes = 8;

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  // splitmix64 finaliser (Steele, Lea, Flood: "Fast splittable pseudorandom number generators")
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

__device__ __forceinline__ int64_t gc_code(const DGcAttr &a, const DCol &c, int64_t r) {
  if (a.kind == 2) {  // bit pattern of an FP32 value
    return (int64_t)(unsigned int)__float_as_uint(__ldg(reinterpret_cast<const float *>(c.p) + r));
  }
  float x;
  int v = 0;
  if (c.dtype == LMFAO_F32) x = __ldg(reinterpret_cast<const float *>(c.p) + r);
  else if (c.dtype == LMFAO_U8) x = (float)(v = __ldg(reinterpret_cast<const unsigned char *>(c.p) + r));
  else x = (float)(v = __ldg(reinterpret_cast<const int *>(c.p) + r));
  if (a.kind == 0) return (int64_t)v;  // a key or categorical value
  int lo = 0, hi = a.nthr;             // bucket: number of thresholds strictly below x
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a.thr + mid) < x) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Group-key part and multiplicity of every join key of relation d.rel toward its parent.
__global__ void gc_view_kernel(DGcRel d, int *err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < d.nrows; r += stride) {
    int64_t k = 0;
    for (int i = 0; i < d.nk; ++i) k += (int64_t)__ldg(reinterpret_cast<const int *>(d.col[d.kcol[i]].p) + r) * d.kstride[i];
    unsigned long long w = 1;
    long long code = 0;
    for (int c = 0; c < d.nchild; ++c) {
      const DGcChild &ch = d.child[c];
      int64_t kk = 0;
      for (int i = 0; i < ch.nk; ++i)
        kk += (int64_t)__ldg(reinterpret_cast<const int *>(d.col[ch.kcol[i]].p) + r) * ch.kstride[i];
      w *= (unsigned long long)ch.cnt[kk];
      code += ch.code[kk];
    }
    if (w == 0) continue;  // no partner in some child: the row does not join
    for (int i = 0; i < d.nattr; ++i) code += gc_code(d.attr[i], d.col[d.attr[i].col], r) * d.attr[i].radix;
    atomicAdd(d.cnt + k, (unsigned long long)w);
    const long long old = (long long)atomicCAS(reinterpret_cast<unsigned long long *>(d.code + k),
                                               (unsigned long long)-1ll, (unsigned long long)code);
    if (old != -1ll && old != code) atomicOr(err, 1);  // a group attribute not determined by the key
  }
}

__device__ __forceinline__ bool table_add(unsigned long long *keys, unsigned long long *cnts, unsigned long long mask,
                                          unsigned long long key, unsigned long long w) {
  unsigned long long h = mix64(key) & mask;
  for (unsigned long long p = 0; p <= mask; ++p) {
    const unsigned long long slot = (h + p) & mask;
    unsigned long long cur = keys[slot];
    if (cur == kEmpty) {
      cur = atomicCAS(keys + slot, kEmpty, key);
      if (cur == kEmpty) cur = key;  // this thread claimed the slot
    }
    if (cur == key) {
      atomicAdd(cnts + slot, w);
      return true;
    }
  }
  return false;  // the table is full
}

// The root pass: one hash update per joined tuple (weighted by its multiplicity).
__global__ void __launch_bounds__(256) gc_root_kernel(DGcRel d, unsigned long long *gkeys, unsigned long long *gcnts,
                                                      unsigned long long gmask, int *err) {
  __shared__ unsigned long long skeys[kCtaSlots];
  __shared__ unsigned long long scnts[kCtaSlots];
  for (int i = threadIdx.x; i < kCtaSlots; i += blockDim.x) {
    skeys[i] = kEmpty;
    scnts[i] = 0ull;
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < d.nrows; r += stride) {
    unsigned long long w = 1;
    long long code = 0;
    for (int c = 0; c < d.nchild; ++c) {
      const DGcChild &ch = d.child[c];
      int64_t kk = 0;
      for (int i = 0; i < ch.nk; ++i)
        kk += (int64_t)__ldg(reinterpret_cast<const int *>(d.col[ch.kcol[i]].p) + r) * ch.kstride[i];
      w *= (unsigned long long)__ldg(ch.cnt + kk);
      code += __ldg(ch.code + kk);
    }
    if (w == 0) continue;
    for (int i = 0; i < d.nattr; ++i) code += gc_code(d.attr[i], d.col[d.attr[i].col], r) * d.attr[i].radix;
    const unsigned long long key = (unsigned long long)code;
    // the CTA's table first, a few probes only
    unsigned int h = (unsigned int)(mix64(key) & (kCtaSlots - 1));
    bool done = false;
    for (int p = 0; p < kCtaProbes && !done; ++p) {
      const unsigned int slot = (h + p) & (kCtaSlots - 1);
      unsigned long long cur = skeys[slot];
      if (cur == kEmpty) {
        cur = atomicCAS(skeys + slot, kEmpty, key);
        if (cur == kEmpty) cur = key;
      }
      if (cur == key) {
        atomicAdd(scnts + slot, w);
        done = true;
      }
    }
    if (!done && !table_add(gkeys, gcnts, gmask, key, w)) atomicOr(err, 4);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kCtaSlots; i += blockDim.x)
    if (skeys[i] != kEmpty && !table_add(gkeys, gcnts, gmask, skeys[i], scnts[i])) atomicOr(err, 4);
}

// Occupied slots of the table -> at most `cap` output groups (codes decoded from the key).
__global__ void gc_compact_kernel(const unsigned long long *gkeys, const unsigned long long *gcnts, int64_t slots,
                                  DGcOut o, unsigned long long *nout) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < slots; s += stride) {
    const unsigned long long key = gkeys[s];
    if (key == kEmpty) continue;
    const unsigned long long pos = atomicAdd(nout, 1ull);
    if ((int64_t)pos >= o.cap) continue;
    unsigned long long rem = key;
    for (int i = 0; i < o.ngb; ++i) {
      o.keys[(int64_t)pos * o.ngb + i] = (int32_t)(unsigned int)(rem / o.radix[i]);
      rem %= o.radix[i];
    }
    o.counts[pos] = (int64_t)gcnts[s];
  }
}

int grid_for_rows(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

void launch_gc_view(const DGcRel &d, int *err, cudaStream_t s) {
  if (d.nrows) gc_view_kernel<<<grid_for_rows(d.nrows), 256, 0, s>>>(d, err);
}

void launch_gc_root(const DGcRel &d, unsigned long long *gkeys, unsigned long long *gcnts, unsigned long long gmask,
                    int *err, cudaStream_t s) {
  if (d.nrows) gc_root_kernel<<<grid_for_rows(d.nrows), 256, 0, s>>>(d, gkeys, gcnts, gmask, err);
}

void launch_gc_compact(const unsigned long long *gkeys, const unsigned long long *gcnts, int64_t slots, const DGcOut &o,
                       unsigned long long *nout, cudaStream_t s) {
  gc_compact_kernel<<<grid_for_rows(slots), 256, 0, s>>>(gkeys, gcnts, slots, o, nout);
}

}  // namespace lmfao
