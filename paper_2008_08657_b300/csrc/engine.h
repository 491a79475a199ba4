// Internal structures of the engine behind include/lmfao.h.
//
// Vocabulary follows Section 2 of the paper: relations joined along a join tree; for
// every edge a directional view V_{u->v} keyed by the join attributes of the edge;
// queries rooted at a node; view groups computed in one pass over the node's relation.
//
// Physical plan (what runs on the GPU). The root relation F (default: the largest) is
// reorganised once at plan time as a two-level trie: its tuples are grouped by the join
// key S of one child (the "segment relation", default: the child with the largest key
// domain), so every segment is a contiguous run of tuples that share their S values
// (Section 2: "the relation ... organised logically as tries"). Children of F whose key
// lies within S are *outer* (looked up once per segment); the others are *inner*
// (looked up once per tuple). Every aggregate is then
//     SUM_seg  psi(seg) * PHI(seg)
// where psi is a product of outer view columns and PHI a per-segment sum of products of
// inner view columns and fact factors -- the alpha/beta decomposition of Fig. 3 with one
// loop level for the segment key and one for the tuple. The per-segment sums PHI are the
// view V_{F->S} from the root to the segment relation.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/lmfao.h"

namespace lmfao {

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define LMFAO_CUDA(call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::lmfao::Error(e_ == cudaErrorMemoryAllocation ? LMFAO_ERR_OOM : LMFAO_ERR_CUDA, \
                           std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

// ---------------------------------------------------------------- relations and batch
struct Column {
  std::string attr;
  int dtype = LMFAO_I32, role = LMFAO_CONT;
  int64_t domain = 0;
  void *dev = nullptr;
  bool owned = false;
};

struct Relation {
  std::string name;
  int64_t nrows = 0;
  std::vector<Column> cols;
  int col(const std::string &a) const {
    for (size_t i = 0; i < cols.size(); ++i)
      if (cols[i].attr == a) return (int)i;
    return -1;
  }
};

struct FactorIn { std::string attr; int fn = 0; int param = 1; };
struct GroupIn { std::string attr; int kind = 0; std::vector<float> thr; };
struct PredIn { std::string attr; int op = 0; float t = 0.f; };
struct QueryIn {
  std::vector<std::vector<FactorIn>> aggs;
  std::vector<GroupIn> gb;
  std::vector<PredIn> filters;
};

// ---------------------------------------------------------------- resolved factors
// A factor of a product: a value factor x^p or an indicator [x op t] (filters are
// indicator factors, so a filtered SUM is the SUM of a longer product).
struct Fac {
  int rel = -1, col = -1;
  int ind = 0;   // 0: value factor, 1: indicator
  int pow = 1;   // value factor exponent
  int op = 0;    // indicator comparison
  float t = 0.f; // indicator threshold
  bool operator<(const Fac &o) const {
    if (rel != o.rel) return rel < o.rel;
    if (col != o.col) return col < o.col;
    if (ind != o.ind) return ind < o.ind;
    if (pow != o.pow) return pow < o.pow;
    if (op != o.op) return op < o.op;
    return t < o.t;
  }
};
using Term = std::vector<int>;  // sorted factor ids

struct GroupItem {
  int rel = -1, col = -1;
  int kind = 0;  // LMFAO_GB_VALUE / LMFAO_GB_BUCKET
  std::vector<float> thr;
  int64_t dom = 1;
  bool operator<(const GroupItem &o) const {
    if (rel != o.rel) return rel < o.rel;
    if (col != o.col) return col < o.col;
    if (kind != o.kind) return kind < o.kind;
    return thr < o.thr;
  }
};

// ---------------------------------------------------------------- views (non-root relations)
struct ViewCol {
  std::vector<int> local;                   // factor ids homed at this relation
  std::vector<std::pair<int, int>> child;   // (child relation, child view column); others: count
  bool integral = true;                     // no value factor anywhere in the subtree term
};
struct CodeSpec {
  int group = -1;       // group item homed here (local code), or -1
  int child_rel = -1;   // else: code taken from this child's view ...
  int child_code = -1;  // ... at this code index
};
struct View {
  int rel = -1, parent = -1;
  std::vector<int> keycols, pkeycols;  // join attributes with the parent (own / parent columns)
  std::vector<int64_t> keydom;
  int64_t nkeys = 1;
  std::vector<ViewCol> cols;  // cols[0]: COUNT
  std::map<Term, int> colmap;
  std::vector<CodeSpec> codes;
  std::map<int, int> codemap;  // group item id -> code index
  std::vector<int> intcol;     // view column -> integral column index (-1 if not integral)
  int nint = 0;
  bool unique_keys = false;    // every key value occurs at most once in the relation
  unsigned int maxmult = 0;    // largest number of tuples sharing one key value
  double count_bound = 1;      // upper bound of the COUNT column (product over the subtree)
  // device storage
  double *v64 = nullptr;      // nkeys x ncols
  float *v32 = nullptr;       // nkeys x ncols (FP32 copy for FP32 passes)
  uint32_t *vint = nullptr;   // nkeys x nint (exact integral columns)
  int32_t *vcodes = nullptr;  // nkeys x ncodes (-1: no tuple)
  int *keyrow = nullptr;      // unique keys: row of each key (-1: none), built at plan time
  int *intcols_dev = nullptr; // view columns copied into vint
};

// ---------------------------------------------------------------- device descriptors
// Limits of the generic kernels (checked by the planner).
constexpr int MAXK = 4;        // key attributes per join key
constexpr int MAXCH = 8;       // children per relation in one view kernel
constexpr int MAXF = 8;        // factors per product part
constexpr int MAXP = 6;        // parts (view columns) per product
constexpr int MAXIN = 6;       // inner children of the root
constexpr int MAXOUT = 6;      // outer children of the root
constexpr int MAXRC = 24;      // root columns read per tuple
constexpr int MAXGR = 4;       // group items per query
constexpr int NB0_MAX = 64;    // per-segment float sums kept in registers
constexpr int NI0_MAX = 8;     // per-segment integral sums kept in registers

struct DFac {       // factor on a column of the relation being scanned
  int col;          // local column slot
  int ind, pow, op;
  float t;
};

struct DViewRef {   // a looked-up view: where its rows are and how to index them
  const double *v64;
  const float *v32;
  const uint32_t *vint;
  const int32_t *codes;
  int ncols, nint, ncodes;
  int nk;
  int kcol[MAXK];        // columns of the scanned relation forming the key
  int64_t kstride[MAXK]; // mixed-radix strides
};

struct DCol {  // a column of the scanned relation
  const void *p;
  int dtype;
};

// One view kernel: scan relation r, look up its children's views, accumulate V_r.
struct DViewKernel {
  int64_t nrows;
  int ncolsin;
  DCol in[MAXRC];
  int nk;
  int kcol[MAXK];
  int64_t kstride[MAXK];
  int nchild;
  DViewRef child[MAXCH];
  // output view
  double *v64;
  int32_t *codes;
  int ncols, ncodes;
  int unique;        // plain stores instead of atomics
  const int *keyrow; // unique keys: row of each key (-1: none); the key-major kernel runs
  int64_t nkeys;
  int nfac;          // factors of all columns (col_fac_off[ncols])
  // columns: [col] -> factor list (offsets into facs) and child column list
  const int *col_fac_off;   // ncols+1
  const DFac *facs;
  const int *col_part_off;  // ncols+1
  const int2 *parts;        // (child index, child column)
  // codes: [code] -> (local column slot, kind, thr offset, nthr) or (child, child code)
  const int4 *code_desc;    // x: local col slot or -1, y: kind, z: thr offset, w: nthr
  const int2 *code_child;   // (child index, child code) when x == -1
  const float *thr;
  int *err;                 // error flags (1: group attribute not determined by the key)
};

// Row-level monomial (product of root-homed, non-segment factors).
struct DMono { int f0, nf; };
// Row term: monomial x product of inner view columns.
struct DRTerm { int mono; int p0, np; int integral; };
struct DPart { int branch, col; };  // branch index and view column (float col or int col)

// Group code source evaluated per segment (outer) or per tuple (inner).
// src: 0 segment key digit (a = digit position); 1 outer view code (a = branch, b = code);
//      2 root column value (a = column slot, kind/thr); 3 inner view code (a = branch, b = code)
struct DGroupRef { int src, a, b, kind, thr0, nthr; int64_t stride; };

// Output items of the combine (B0: per-segment PHI column; B1: grouped PHI block).
struct DCombItem {
  int psi;          // outer term id
  int block;        // -1: B0, else B1 set index
  int col;          // column within the block (float or int according to integral)
  int integral;
  int og0, nog;     // outer group refs
  int ig0, nig;     // inner group refs (B1: in the set's digit order, with the query strides)
  int64_t out;      // base cell of the query output (float: fsum index; int: icnt index)
  int64_t cellmul;  // multiplier from cell index to the output array index
  int yint;         // B1: the column is an integral (count) column
  int sel;          // B1: filter index the entry reads (-1: every group code)
};

// Outer term: segment-key factors x product of outer view columns.
struct DPsi { int f0, nf; int p0, np; int integral; };
struct DSegFac { int digit; int pow; int ind, op; float t; };

}  // namespace lmfao
