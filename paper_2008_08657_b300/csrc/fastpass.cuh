// Specialised root pass for plans with at most one inner child of the root.
//
// Per tuple r of segment s (Fig. 3 with two loop levels, segment key outside, tuple inside):
//   u_j(r)  monomials over the root's own attributes (j < nm),
//   v_w(r)  the inner view row V_I[k_I(r)] restricted to the nw columns the batch needs,
//   B0:     PHI0[s][j][w]  += u_j * v_w                 (registers; warp sum per work item)
//   B1:     PHI1[s][g][c]  += u_j(c) * v_w(c)          (per-warp shared histogram per segment,
//                                                       g = inner group code of the tuple)
//   B3:     P[k_I][c]      += w_s * u_j(c)             (CTA-private shared partials; this is the
//                                                       view from the root to the inner relation,
//                                                       V_{S->I} of Fig. 2, w_s the outer weight)
#pragma once

#include "kernels.cuh"

namespace lmfao {

constexpr int FMAXM = 16;   // monomials
constexpr int FMAXW = 8;    // inner view columns
constexpr int FMAXF = 24;   // factors of all monomials
constexpr int FMAXB1 = 4;   // B1 group sets
constexpr int FMAXC = 8;    // columns per B1 set / B3 columns
constexpr int FMAXX = 6;    // root columns read per tuple (fact values and group columns)
constexpr int FMAXFAM = 16; // filters of a filter family (disjoint conjunctions, e.g. tree leaves)
constexpr int FMAXBIT = 32; // distinct predicates of a filter family
constexpr int FMAXB4 = 256; // items accumulated per CTA without segments

struct DFastB1 {
  int G;                 // cells of the group set
  int nref;              // group refs (src 2: root column slot; src 3: inner view code)
  DGroupRef ref[2];      // stride = radix inside the set
  int nf, ni;            // float / integral columns
  int fj[FMAXC], fw[FMAXC];
  int ij[FMAXC], iw[FMAXC];
  int smem_f, smem_i;    // offsets of this set inside a warp's histogram (floats / u32)
  // refs of src 4 read the tuple's filter index
  int64_t gbase_f, gbase_i;  // offsets in phi1f / phi1i (per segment: G x nf / G x ni)
};

struct DFast {
  int64_t nwork;
  const DWork *work;
  const int *work_q;      // tuple quantiles of the work list (kWorkQ + 1 entries)
  const unsigned long long *wseg;
  int ncols;
  DCol col[MAXRC];
  // inner branch
  int ni;                 // 0 or 1
  int nk;
  int kslot[2];
  int64_t kstride[2];
  int64_t nkeys;
  int nw;                 // inner view columns used (column 0: COUNT)
  int ncode;              // inner view codes used (B1 / B3 groups)
  const void *table;      // [nkeys][nw] in T (prepared by fast_prep_kernel)
  const int *codes;       // [nkeys][ncode]
  int smem_view;          // stage table and codes in shared memory
  // monomials: u_j = prod_i x_i^mexp[j][i] * prod of the indicators of monomial j
  int nm;
  int nx;                 // root columns whose values feed the monomials
  int xslot[FMAXX];
  unsigned char mexp[FMAXM][FMAXX];
  int nind;               // indicator factors on root columns
  DFac ind[FMAXF];
  int ind_mono[FMAXF];
  // B0
  void *phi0f;            // [nseg][nm*nw]
  unsigned long long *phi0i;  // [nseg][n0i]
  int n0i;
  int i0j[NI0_MAX], i0w[NI0_MAX];
  // B1
  int nb1;
  DFastB1 b1[FMAXB1];
  int hist_f, hist_i;     // per-warp histogram sizes (floats, u32)
  float *phi1f;
  unsigned int *phi1i;
  int64_t phi1f_seg, phi1i_seg;  // per-segment stride
  // B3
  int n3;
  int j3[FMAXC];
  int int3[FMAXC];
  int smem_p;             // P in shared memory (else global atomics)
  int n3f, n3i;           // float / integral B3 columns (P columns are split by kind)
  int p3col[FMAXC];       // B3 column -> index within its kind
  unsigned int *ticket;   // work-item ticket (zeroed before every launch)
  // lean variant: monomials are the full basis of degree <= 2 over the nx value columns
  // (1, x_i, x_i x_j), no indicators, B1 columns are inner COUNTs only
  int lean;
  int vec;                // root columns padded by 16 bytes: 4-tuple vector loads
  int lanes;              // generated pass: one tuple per lane and step (coalesced 4-byte loads)
                          // instead of a 4-tuple quad per lane (16-byte loads, ragged head/tail)
  int b1code[FMAXB1];     // inner view code (position in codes) of each B1 set
  double *p3f;            // [nkeys][n3]
  unsigned long long *p3i;
  float *p3f32;           // FP32 partials when P is not in shared memory (global atomics)
  const float *thr;
  // filter family: the tuple's filter index ("leaf") from predicate bits
  int nfam;                       // 0: no family
  unsigned int fmask[FMAXFAM];    // predicate bits of each filter
  int nob;                        // predicates on outer relations (one bit each)
  int obit_outer[FMAXBIT], obit_col[FMAXBIT], obit_pos[FMAXBIT];
  int ibit_code;                  // inner predicate bits: codes column index (-1: none)
  int nrb;                        // predicates on root columns
  DFac rb[FMAXBIT];
  int rb_pos[FMAXBIT];
  int nouter;
  DOuter outer[MAXOUT];
  DSegment seg;
  int b3leaf;                     // B3 partials split by filter index (1: not split)
  // B4: items accumulated per CTA (no outer dependency, row-level groups)
  int nb4;
  int b4_off[FMAXFAM + 2];            // B4 items of filter index f: [b4_off[f+1], b4_off[f+2]); -1 first
  int b4_j[FMAXB4], b4_w[FMAXB4], b4_int[FMAXB4], b4_sel[FMAXB4];
  int b4_g0[FMAXB4], b4_ng[FMAXB4];   // group refs (src 2) in grefs4
  int b4_so[FMAXB4];                  // shared-memory output base
  int64_t b4_cellmul[FMAXB4];
  const DGroupRef *grefs4;
  int b4_fcells, b4_icells;
  int nb4mirror;
  const DMirror *b4mirror;
  double *fsum;
  unsigned long long *icnt;
};

void launch_fast_prep(const DFast &d, const double *v64, int vcols, const int *wcol, const int32_t *vcodes,
                      int vncodes, const int *codecol, void *table, int *codes, bool fp64, cudaStream_t s,
                      const int2 *ib, int nib);
size_t fast_smem(const DFast &d, bool fp64, int block);
bool launch_fast_pass(const DFast &d, bool fp64, int grid, int block, cudaStream_t s);
bool fast_shape_ok(int nm, int nw);  // a kernel variant exists for nm monomials x nw view columns
bool lean_shape_ok(int nx, int nw);

// B3 finalisation: out[cell(k)] += V[k][w] * P[k][c] over the inner relation's keys.
struct DB3Item {
  int w;          // view column (FP64 view)
  int c;          // P column (within the float or integral part)
  int leaf;       // filter index of a filter family (-1: none)
  int integral;
  int pint;       // the P column is integral (also for a float item)
  int ig0, nig;   // group refs (src 3: view code index)
  int64_t out, cellmul;
};
struct DB3Final {
  int64_t nkeys;
  const double *v64;
  int vcols;
  const int32_t *vcodes;
  int vncodes;
  const double *p3f;
  const unsigned long long *p3i;
  const float *p3f32;     // used instead of p3f when non-null
  int n3;
  int n3f, n3i;
  int nitems;
  const DB3Item *items;
  const DGroupRef *grefs;
  double *fsum;
  unsigned long long *icnt;
};
void launch_b3_final(const DB3Final &d, cudaStream_t s);

}  // namespace lmfao
