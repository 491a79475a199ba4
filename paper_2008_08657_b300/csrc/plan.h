// Planner state of a context (join tree, logical views and groups, physical plan).
#pragma once

#include <array>
#include <set>

#include "codegen.h"
#include "fastpass.cuh"

namespace lmfao {

size_t fact_pass_smem(const DFactPass &d, bool fp64, int block);

// Join tree over the relations (Section 2 "the backbone of this plan is a join tree").
struct JoinTree {
  int root = -1;
  std::vector<int> parent;                 // -1 for the root
  std::vector<std::vector<int>> children;
  std::vector<int> depth;
  std::vector<int> post;                   // non-root relations, children before parents
};

// Logical plan of Section 2: per-query roots, directional views after merging, groups.
struct LogicalView {
  int from = -1, to = -1;
  std::vector<std::string> key;            // join attributes of the edge + carried group-by attributes
  std::set<std::string> aggs;              // aggregate parts over the subtree (canonical strings)
  std::set<int> queries;
  std::set<int> deps;                      // incoming views it is computed from
};
struct LogicalGroup {
  int node = -1;
  std::vector<int> views;                  // outgoing views computed by the group
  std::vector<int> queries;                // queries whose root is the node
  std::set<int> deps;                      // groups it depends on
};
struct LogicalPlan {
  std::vector<int> query_root;
  std::vector<LogicalView> views;
  std::vector<LogicalGroup> groups;
};

struct QueryOut {
  int64_t cells = 1;
  int64_t fo = 0, io = 0;  // offsets into fsum (cells x naggs) and icnt (cells x (1 + naggs))
  int naggs = 0;
  std::vector<int64_t> dom;
  std::vector<int> integral;
  std::vector<int> gitems;  // group item ids in query order
};

struct DeviceArena {  // allocations owned by a plan
  std::vector<void *> ptrs;
  void *alloc(size_t bytes);
  template <typename T> T *upload(const std::vector<T> &v, cudaStream_t s);
  void release();
};

struct PhysPlan {
  bool fp64 = false;
  bool split_bf16 = false;         // dense block contraction as split BF16 on the tensor cores
  int mode = LMFAO_MODE_FACTORISED;
  int root = -1, segrel = -1;
  std::vector<int> segcols;        // root columns forming the segment key
  std::vector<int64_t> segdom;
  int64_t nseg = 1;
  int prefix_len = 0;              // leading segment digits forming the block key of the combine
  std::vector<int> outer, inner;   // root children
  std::vector<int> kind;           // per relation: 0 root, 1 outer subtree, 2 inner subtree
  std::vector<int> branch;         // per relation: root child whose subtree holds it (-1 root)
  std::vector<View> views;         // per relation (root entry unused)
  std::vector<Fac> facs;
  std::map<Fac, int> facmap;
  std::vector<GroupItem> gitems;
  std::map<GroupItem, int> gmap;
  std::vector<QueryOut> qout;
  int64_t nfsum = 0, nicnt = 0;
  // root tuple level
  std::vector<int> rowcols;        // root columns read per tuple
  std::map<int, int> rowslot;
  std::vector<std::vector<int>> monos;
  std::map<std::vector<int>, int> monomap;
  struct RT { int mono; std::vector<std::pair<int, int>> parts; bool integral; };
  std::vector<RT> rts;
  std::map<std::pair<int, std::vector<std::pair<int, int>>>, int> rtmap;
  struct Psi { std::vector<int> segf; std::vector<std::pair<int, int>> parts; bool integral; };
  std::vector<Psi> psis;
  std::map<std::pair<std::vector<int>, std::vector<std::pair<int, int>>>, int> psimap;
  std::vector<int> b0f, b0i;       // row terms summed per segment
  std::vector<DCombItem> comb;
  std::vector<DB2Item> b2;
  std::vector<DGroupRef> grefs;
  std::vector<float> thr;
  int nb0 = 4;
  // specialised root pass (at most one inner child)
  struct Fast {
    bool on = false;
    bool lean = false;                         // lean kernel variant (degree <= 2 basis)
    std::vector<int> lean_cols;                // value columns of the basis
    std::vector<std::vector<int>> monos;       // row factor lists
    std::vector<int> wcols;                    // inner view columns (0: COUNT)
    std::vector<std::pair<int, int>> int0;     // integral (monomial, column) pairs of PHI0
    struct B1 {
      std::vector<DGroupRef> refs;
      std::vector<std::vector<float>> thrs;
      std::vector<int64_t> dom;
      int64_t G = 1;
      std::vector<std::pair<int, int>> fcols, icols;
    };
    std::vector<B1> b1;
    std::vector<std::pair<int, bool>> p3;      // B3 columns: (monomial, integral)
    std::vector<DB3Item> b3;
    int b3leaf = 1;                            // B3 partials split by filter index
    struct B4 {                                // CTA-private items (no outer dependency)
      int j, w, integral, sel, q;
      std::vector<DGroupRef> refs;
      int64_t out, cellmul;
    };
    std::vector<B4> b4;
    int fam_k = 0;                             // filter family
    std::vector<unsigned int> fmask;
    struct Bit { int a, pos, fac; };           // outer: (outer idx, view col, bit); inner: (view col, bit)
    std::vector<Bit> obits_;
    std::vector<std::array<int, 3>> obits, ibits, rbits;
  } fast;
  DFast fd{};
  DB3Final b3f{};
  int *fwcol_dev = nullptr, *fcodecol_dev = nullptr;
  int2 *fibits_dev = nullptr;
  int fnibits = 0;
  int fast_grid = 0, fast_block = 512;
  GenRootPass gen;                 // plan-specialised root pass (null: the template kernel)
  std::vector<DB1Set> b1sets;
  // device
  DeviceArena arena;
  std::vector<DCol> rowdev;        // reorganised root columns (per row slot)
  DWork *work = nullptr;
  int *work_q = nullptr;           // tuple quantiles of the work list (CTA ranges)
  int64_t nwork = 0;
  unsigned long long *wseg = nullptr;
  void *phi0f = nullptr;
  unsigned long long *phi0i = nullptr;
  double *fsum = nullptr;
  unsigned long long *icnt = nullptr;
  int *err = nullptr;
  std::vector<DViewKernel> vk;     // per view relation, in post order
  std::vector<int> vk_rel;
  std::vector<GenView> vgen;       // per view: the generated kernel (null fn: a built-in one runs)
  DFactPass fp{};
  DCombine cb{};
  DComb2 c2{};
  int c2_grid = 0, c2_block = 512;
  std::vector<DEntry> c2h_ent;     // host copies of the entry combine's entries and outer-cell sets
  std::vector<int> c2h_og_off;
  std::vector<DGroupRef> c2h_og_refs;
  DComb4 c4{};                     // projection combine (two-digit segment keys)
  bool use_c4 = false;
  DComb3 c3{};
  bool use_c3 = false, no_c3 = false;
  DComb5 c5{};                     // two-kernel block combine (combine5.cu)
  bool use_c5 = false;
  std::vector<int2> c3_bsrc;       // per B term (outer view, column), (-1, -1) for 1; empty when
                                   // some B term is a product or has a segment-digit factor
  std::string c5_why;              // why the two-kernel block combine does not run (if not)
  std::string fast_why;            // why the specialised root pass declined the batch (if it did)
  std::map<int, int *> result_flags;  // per query: integral flags on the device (lmfao_result_device)
  int c3_grid = 0, c3_block = 512;
  DSegWeight sw{};
  int fp_grid = 0, fp_block = 256;
  std::vector<std::string> kernel_names;
  double plan_ms = 0;
  double reorg_ms = 0;             // host wall time of reorganising the root relation in this plan
  std::vector<int64_t> seg_hist;   // tuples per segment of the root relation
  int work_chunk = 4096;           // tuples per work item of the root pass (a tile the tuner picks)
  bool tuned = false, tune_cached = false;  // tiles chosen by the autotuner (from its cache file)
  int tune_candidates = 0;         // launch shapes timed by the autotuner
  double tune_ms = 0;              // host time spent autotuning
  bool reorg_cached = false;       // the segment order came from an earlier plan
};

}  // namespace lmfao

struct lmfao_ctx;
namespace lmfao {
// Words per CART query descriptor: icnt base, fsum base, buckets, aggregates, index of SUM(y),
// index of SUM(y^2).
constexpr int kCartDescWords = 6;
// Checks the arguments of a CART split-variance call (Section 3, decision trees) against the
// context's last run: every query id valid, one BUCKET group-by, exactly three aggregates that
// are COUNT, SUM(y) and SUM(y^2) of one attribute y (in any order), and the same number of
// buckets for all queries. Writes n descriptors of kCartDescWords words into desc (host, may
// be null) and returns the bucket count; *plan (may be null) receives the physical plan that
// holds the queries (all of them must be evaluated by one plan). Throws Error(LMFAO_ERR_ARG /
// ERR_NOT_PLANNED / ERR_UNSUPPORTED).
int cart_descriptors(lmfao_ctx *ctx, const int *qids, int n, int64_t *desc, PhysPlan **plan);
}  // namespace lmfao
