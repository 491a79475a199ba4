// Device-side descriptors and launchers shared by the host planner and the kernels.
#pragma once

#include "engine.h"

namespace lmfao {

// Root fact pass (Section 2 multi-output plan for the root group; Fig. 3 with the segment
// key as the outer trie level): one warp per work item (a contiguous run of tuples of one
// segment). Per tuple: inner view lookups, row terms; per segment: sums of the B0 row
// terms (the view V_{F->S}); per tuple: direct accumulation of B2 items.
struct DB2Item {
  int psi;       // outer term id
  int rterm;     // row term id
  int integral;
  int og0, nog;  // outer group refs (segment level)
  int ig0, nig;  // inner group refs (tuple level)
  int64_t out;   // output base index (fsum or icnt)
  int64_t cellmul;
};

struct DWork {  // one work item: tuples [r0, r0 + len) of segment seg
  long long r0;
  int seg;
  int len;
};
// Tuple quantiles of the work list: entry j (0 <= j <= kWorkQ) is the first item whose first
// tuple is at or past j / kWorkQ of all tuples, so CTA b of G takes the items
// [q[kWorkQ b / G], q[kWorkQ (b + 1) / G]): contiguous ranges of about equal tuple counts.
constexpr int kWorkQ = 4096;

struct DOuter {  // an outer child: key index from the segment id
  DViewRef v;
  int64_t dstride[8];  // contribution of each segment digit to the view key index
};

struct DSegment {  // segment key decoding
  int ndig;
  int64_t dom[8];
  int64_t radix[8];  // seg = sum digit_i * radix[i]
};

struct DFactPass {
  int64_t nwork;
  const DWork *work;
  const unsigned long long *wseg;  // outer count product per segment
  int ncols;
  DCol col[MAXRC];
  int ninner;
  DViewRef inner[MAXIN];
  int nmono;
  const DMono *mono;
  const DFac *facs;
  int nrt;
  const DRTerm *rt;
  const DPart *parts;
  int n0f, n0i;               // B0 float terms = row terms b0f[0..n0f), int = b0i[..]
  const int *b0f, *b0i;
  void *phi0f;                // n_seg x n0f (float or double)
  unsigned long long *phi0i;  // n_seg x n0i
  // B2
  int nb2;
  const DB2Item *b2;
  const DGroupRef *grefs;
  const float *thr;
  // outer side for B2 psi / outer group codes
  DSegment seg;
  int nouter;
  DOuter outer[MAXOUT];
  int npsi;
  const DPsi *psi;
  const DSegFac *segfacs;
  const DPart *psiparts;
  double *fsum;
  unsigned long long *icnt;
  int b2_smem_items;  // B2 items whose psi is staged per warp
};

// A query output region mirrored in shared memory by the combine (CTA-private sums).
struct DMirror { long long gout; int soff; int len; int integral; int pad; };

// A B1 block of per-segment sums grouped by inner group codes.
struct DB1Set {
  int G, nref;
  int64_t radix[2], dom[2];
  int nf, ni;
  int64_t gbase_f, gbase_i;
};

// What every combine reads: the segments and their outer views, the outer terms psi, the
// per-segment sums PHI0 / PHI1 and the outputs (the block, projection and entry combines take
// their own descriptors from it).
struct DCombine {
  int64_t nseg;
  const unsigned long long *wseg;
  DSegment seg;
  int nouter;
  DOuter outer[MAXOUT];
  int npsi;
  const DPsi *psi;
  const DSegFac *segfacs;
  const DPart *psiparts;
  int n0f, n0i;
  const void *phi0f;
  const unsigned long long *phi0i;
  const DGroupRef *grefs;
  const float *thr;
  int nsets;
  const DB1Set *sets;
  const float *phi1f;
  const unsigned int *phi1i;
  int64_t phi1f_seg, phi1i_seg;
  double *fsum;
  unsigned long long *icnt;
};

// One output entry of the combine: psi term x one Y column, written to
// out + (outer cell + icell) * cellmul.
struct DEntry {
  int psi, ycol, og, integral, so, yint;
  long long out, cellmul, icell;
};

struct DComb2 {
  int64_t nseg;
  const unsigned long long *wseg;
  DSegment seg;
  int nouter;
  DOuter outer[MAXOUT];
  int nstage;
  const int2 *stage_col;  // (outer view, column) staged per segment
  int npsi;
  const DPsi *psi;
  const DSegFac *segfacs;
  const int *psi_stage;   // psi parts -> staged column
  int nog;
  const int *og_off;      // outer-cell sets (CSR over grefs)
  const DGroupRef *grefs;
  int n0f, n0i, nyf, nyi;
  const void *phi0f;
  const unsigned long long *phi0i;
  const float *phi1f;
  const unsigned int *phi1i;
  int64_t phi1f_seg, phi1i_seg;
  int nent;
  const DEntry *ent;
  int nmirror;
  const DMirror *mirror;
  int mirror_f, mirror_i;
  double *fsum;
  unsigned long long *icnt;
  int tile;
};
size_t combine2_smem(const DComb2 &d, bool fp64);
void launch_combine2(const DComb2 &d, bool fp64, int grid, int block, cudaStream_t s);

// Projection combine for a two-digit segment key (major digit d0, minor digit d1; segment =
// d0 * dom1 + d1). An entry SUM_s psi(s) * Y_c(s) into cell og(s) is classified by the
// digits its outer term and outer cells depend on:
//   class 0 (none):  psi = 1, one cell: SUM_s Y_c(s);
//   class 1 (d0):    SUM_d0 psi(d0) * Yd0[d0][c],  Yd0[d0][c] = SUM_d1 Y_c(d0, d1);
//   class 2 (d1):    SUM_d1 psi(d1) * Yd1[d1][c],  Yd1[d1][c] = SUM_d0 Y_c(d0, d1);
//   class 3 (both):  per segment.
// The projections Yd0 / Yd1 are the views from the root to the outer relations keyed by one
// digit (Fig. 2's views toward other roots); every Y column is streamed once per projection
// and the entries then read only the small projections. Sums run over the segments whose
// outer partners all exist (w_s != 0); float columns are projected in FP64, integral ones in
// INT64.
struct DEntry4 {
  int psi, og, cls, flags;  // psi: column of the class's term table; og: the outer-cell set;
                            // flags: 1 integral output, 2 integral Y column
  int job, tog;             // Y column job; column of the class's cell table
  int sbase, pad;           // class 3: first slot in the CTA's slots of the entry's tile
  long long out, cellmul, icell;
};
// Outer terms and cells of one entry class, tabulated per value of its digit(s): terms in
// FP64 and exactly (integral terms), cells as compact indices over the cell set's attributes.
struct DTab4 {
  int nt, ng;               // tabulated terms and cell sets
  const int *t, *g;         // their ids
  double *pf;               // classes 1, 2: [nt][nvalues] (lanes over the digit read consecutive
  unsigned long long *pi;   // words); class 3: [nvalues][nt] (a segment's terms together)
  long long *cell;          // the same with ng (-1: a code is missing, or class 3 and w_s = 0)
};
struct DComb4 {
  DComb2 c;                 // segments, outer views, psi terms, outer-cell sets, Y columns
  int dom0, dom1;
  int njobs;
  const int2 *job;          // (integral Y column, column index within its kind)
  const DEntry4 *ent;       // entries of classes 0..2
  int nent012;
  int nent3;
  const DEntry4 *ent3;      // class 3 entries, grouped by job: job j has [e3_off[j], e3_off[j+1])
  const int *e3_off;
  DTab4 tab[4];             // classes 1 (per d0), 2 (per d1), 3 (per segment); [0] unused
  int max_slots3;           // shared slots of one tile of 256 class 3 entries
  double *yd0_f, *yd1_f, *yall_f;             // [njobs][dom0], [njobs][dom1], [njobs]
  unsigned long long *yd0_i, *yd1_i, *yall_i;
  int need_d0, need_d1;
  int skip_counts;          // every outer COUNT is 0 or 1: on live segments the COUNT parts of
                            // an outer term are 1 and are left out of it
  const long long *og_ncells;                 // per outer-cell set: compact cells
  const long long *og_cstride, *og_dom;       // per outer group ref: compact stride and domain
  int max_cells;
  // streaming form (stream != 0): one pass over the per-segment sums in tiles of c1 minor x
  // c0 major digit values (grid nx x ny) forms partial projections (Yd0p: nx x dom0 x njobs,
  // Yd1p: ny x dom1 x njobs, 8-byte words typed by the job) and, when fused3, the class 3
  // entries from the staged rows (slots: the cumulative cell base of each entry in pad)
  int stream, c1, c0, nx, ny, sblock, fused3, nslots3;
  unsigned long long *yd0p, *yd1p;
};
void launch_combine4(const DComb4 &d, bool fp64, cudaStream_t s);

struct DSegWeight {
  int64_t nseg;
  DSegment seg;
  int nouter;
  DOuter outer[MAXOUT];
  unsigned long long *wseg;
};

// launchers (kernels.cu)
void launch_view_kernel(const DViewKernel &d, cudaStream_t s);
void launch_view_finish(const double *v64, float *v32, uint32_t *vint, const int *intcols,
                        int ncols, int nint, int64_t nkeys, int *err, cudaStream_t s);
void launch_segment_weights(const DSegWeight &d, cudaStream_t s);
void launch_fact_pass(const DFactPass &d, bool fp64, int nb0, int grid, int block, cudaStream_t s);
void launch_segment_ids(const DCol *cols, int ncols, const int64_t *radix, int64_t n, int *segid,
                        cudaStream_t s);
void launch_histogram(const int *segid, int64_t n, unsigned int *hist, cudaStream_t s);
void launch_scatter_rows(const int *segid, int64_t n, unsigned long long *cursor, const DCol *in,
                         DCol *out, const int *elem_size, int ncols, unsigned int *dest, cudaStream_t s);
void launch_permute_rows(const unsigned int *dest, int64_t n, const DCol *in, DCol *out, const int *elem_size,
                         int ncols, cudaStream_t s);
void launch_range_check(const void *p, int dtype, int64_t n, int64_t domain, int *bad, cudaStream_t s);
// Views of unique-key relations computed key by key (kVkb keys per CTA, a shared tile of their
// rows): used when the tile fits 48 KB of shared memory.
constexpr int kVkb = 128;
size_t view_key_rows_smem(const DViewKernel &d);
void launch_key_rows(const DCol *cols, int ncols, const int64_t *stride, int64_t n, int *keyrow, cudaStream_t s);
void launch_key_multiplicity(const DCol *cols, int ncols, const int64_t *stride, int64_t n,
                             unsigned int *hist, cudaStream_t s);
void launch_max_u32(const unsigned int *h, int64_t n, unsigned int *out, cudaStream_t s);
void launch_cart_variances(const unsigned long long *icnt, const double *fsum, const int64_t *qdesc,
                           int n, int nb_max, double *out, cudaStream_t s);
void launch_cart_split(const unsigned long long *icnt, const double *fsum, const int64_t *qdesc, const int *qbeg,
                       int nnodes, int2 *best, double *score, double *stats, cudaStream_t s);
void launch_ridge(const unsigned long long *icnt, const double *fsum, int64_t io, int64_t fo, const int *zmap, int d,
                  double lambda, int method, int iters, double step, double *out, cudaStream_t s);
void launch_results(const unsigned long long *icnt, const double *fsum, int64_t cells, int naggs,
                    const int *integral, int64_t *counts, double *sums, cudaStream_t s);

}  // namespace lmfao

namespace lmfao {

// Prefix-block combine. The segment key is ordered so that its first L digits (the
// prefix) are the key of the "A" outer views; the other outer views ("B") vary inside a
// block of m consecutive segments sharing a prefix. Every outer term factors as
// psi_t(s) = a_alpha(p) * b_beta(s) (Fig. 3 with the prefix as one more loop level), so
//     SUM_s psi_t(s) Y_c(s) = SUM_p a_alpha(p) * Z_p[beta][c],   Z_p = B_p^T Y_p,
// a contraction over the m segments of block p, computed once per block for all
// (beta, c), followed by one multiply-add per output entry and block.
struct DEntry3 {
  int a, b, c, yint, integral, og, so, pad;
  long long out, cellmul, icell;
};

struct DComb3 {
  int64_t nblocks, m;
  const unsigned long long *wseg;
  DSegment seg;
  int nouter;
  DOuter outer[MAXOUT];
  int nbst, nb, nbi;        // staged B columns, B terms, integral B terms (first nbi terms)
  int nbpart;               // entries of bpart
  const int2 *bstage;       // (outer view, column)
  const DPsi *bterm;        // parts index bpart[]
  const int *bpart;         // -> staged B column
  int nast, na;
  const int2 *astage;
  const DPsi *aterm;
  const int *apart;
  const DSegFac *segfacs;   // digits < L belong to A terms, others to B terms
  int n0f, n0i, nyf, nyi;   // Y columns: float [0, nyf), integral [0, nyi)
  const void *phi0f;
  const unsigned long long *phi0i;
  const float *phi1f;
  const unsigned int *phi1i;
  int64_t phi1f_seg, phi1i_seg;
  int nog;
  const int *og_off;
  const DGroupRef *grefs;   // A-level refs (src 0 digit < L, or src 1 A view)
  int nent;
  const DEntry3 *ent;
  int nmirror;
  const DMirror *mirror;
  int mirror_f, mirror_i;
  double *fsum;
  unsigned long long *icnt;
};
size_t combine3_smem(const DComb3 &d, bool fp64);
void launch_combine3(const DComb3 &d, bool fp64, int grid, int block, cudaStream_t s);

// Two-kernel prefix-block combine (combine5.cu): block_z_kernel computes per block p the
// contraction Z_p = B_p^T Y_p (FP32 or FP64 on the CUDA cores, or split-BF16 on the tensor
// cores), the integral part exactly, the A terms a_alpha(p) and the outer cells, into global
// scratch arrays; block_entries_kernel then forms SUM_p a_alpha(p) Z_p[beta][c] per entry.
struct DComb5 {
  DComb3 c;                  // segments, outer views, A/B terms, Y columns, entries, outputs
  int kc;                    // segments per chunk (a multiple of 16 on the tensor-core path)
  int npad;                  // tensor-core path: N of the MMA (B terms rounded up to 16)
  int tmem_cols;             // tensor-core path: tensor-memory columns allocated per CTA
  int tc;                    // 1: contraction on the tensor cores (split BF16)
  int dense;                 // 1: every B term is one outer-view column or 1 (block_zd_kernel)
  int pipe;                  // dense with every B column from outer view bout, whose row for
  int bout;                  // segment j of a block is the block's row + j x bstride
  int64_t bstride;           // (block_zp_kernel)
  const int2 *bsrc;          // dense: per B term (outer view, column); (-1, -1) for the constant 1
  int bulk;                  // 1: per-segment sums staged with TMA bulk copies (16-byte aligned)
  int grid;                  // CTAs of block_z_kernel
  int eranges;               // block ranges of block_entries_kernel (grid.y)
  void *z;                   // nblocks x nb x ny (FP32 or FP64)
  unsigned long long *zi;    // nblocks x nbi x nyi
  void *a;                   // nblocks x na
  unsigned long long *ai;    // nblocks x na (integral A terms)
  long long *cells;          // nblocks x nog (-1: a code of the cell is missing)
  int *live;                 // nblocks: some segment of the block has all its outer partners
  int *err;                  // error flags (8: a bounded wait of block_z_kernel ran out)
};
size_t combine5_smem(const DComb5 &d, bool fp64);
bool combine5_dense_fits(const DComb3 &d);  // the dense kernel's register tiles cover Z_p
void launch_combine5_z(const DComb5 &d, bool fp64, cudaStream_t s);
void launch_combine5_entries(const DComb5 &d, bool fp64, cudaStream_t s);

// COUNT GROUP BY with hash-table results (sparse.cu).
constexpr int GC_MAXATTR = 16;   // group attributes
constexpr int GC_MAXCOL = 32;    // columns of a relation visible to the kernels
struct DGcAttr {                 // a group attribute homed at the relation being scanned
  int kind;                      // 0: key / categorical value, 1: bucket, 2: FP32 bit pattern
  int col, nthr;
  const float *thr;
  int64_t radix;                 // weight of its code in the group key
};
struct DGcChild {                // the partial view of a child relation
  int nk;
  int kcol[MAXK];
  int64_t kstride[MAXK];
  const unsigned long long *cnt; // multiplicity per join key
  const long long *code;         // group-key part per join key (-1: no row)
};
struct DGcRel {
  int64_t nrows;
  DCol col[GC_MAXCOL];
  int nk;                        // the join key toward the parent (non-root relations)
  int kcol[MAXK];
  int64_t kstride[MAXK];
  int nchild;
  DGcChild child[MAXCH];
  int nattr;
  DGcAttr attr[GC_MAXATTR];
  unsigned long long *cnt;       // output partial view (non-root relations)
  long long *code;
};
struct DGcOut {
  int ngb;
  int64_t radix[GC_MAXATTR];
  int64_t cap;
  int32_t *keys;                 // cap x ngb group codes
  int64_t *counts;               // cap
};
void launch_gc_view(const DGcRel &d, int *err, cudaStream_t s);
void launch_gc_root(const DGcRel &d, unsigned long long *gkeys, unsigned long long *gcnts, unsigned long long gmask,
                    int *err, cudaStream_t s);
void launch_gc_compact(const unsigned long long *gkeys, const unsigned long long *gcnts, int64_t slots, const DGcOut &o,
                       unsigned long long *nout, cudaStream_t s);

}  // namespace lmfao
