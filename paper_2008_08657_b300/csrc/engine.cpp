// Host side of the engine: the C ABI of include/lmfao.h, the planner (join tree, view
// generation, multi-output plan) and the executor that enqueues the kernels.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <fstream>
#include <sys/stat.h>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <sstream>

#include "ctx.h"
#include "fastpass.cuh"

namespace lmfao {
int64_t mlp_param_count(int d);
}
extern "C" int lmfao_mlp_forward(const float *x, int n, int d, const float *params, float *h1, float *h2, float *y,
                                 void *stream);

using namespace lmfao;


namespace lmfao {

void *DeviceArena::alloc(size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(LMFAO_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  ptrs.push_back(p);
  return p;
}

template <typename T>
T *DeviceArena::upload(const std::vector<T> &v, cudaStream_t s) {
  T *p = (T *)alloc(v.size() * sizeof(T));
  if (!v.empty()) LMFAO_CUDA(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return p;
}

void DeviceArena::release() {
  for (void *p : ptrs) cudaFree(p);
  ptrs.clear();
}

}  // namespace lmfao

namespace {

int fail(lmfao_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

template <typename F>
int guarded(lmfao_ctx *ctx, F &&f) {
  if (!ctx) return LMFAO_ERR_ARG;
  try {
    ctx->last_error.clear();
    if (ctx->device >= 0) cudaSetDevice(ctx->device);
    return f();
  } catch (const Error &e) {
    return fail(ctx, e.code, e.what());
  } catch (const std::exception &e) {
    return fail(ctx, LMFAO_ERR_ARG, e.what());
  }
}

void drop_plan(lmfao_ctx *ctx) {
  if ((ctx->plan || !ctx->subs.empty()) && ctx->device >= 0) {
    cudaStreamSynchronize(ctx->stream);
    if (ctx->run_stream) cudaStreamSynchronize(ctx->run_stream);
  }
  if (ctx->plan && ctx->device >= 0) {
    ctx->plan->arena.release();
    delete ctx->plan;
    ctx->plan = nullptr;
  }
  for (auto &sp : ctx->subs) {
    sp.plan->arena.release();
    delete sp.plan;
  }
  ctx->subs.clear();
  ctx->qroute.clear();
  ctx->planned = ctx->ran = false;
}

// The physical plan that evaluates batch query q and q's index in it (a batch with several
// roots has one plan per root); nullptr when there is no plan.
std::pair<PhysPlan *, int> plan_of(lmfao_ctx *ctx, int q) {
  if (ctx->plan) return {ctx->plan, q};
  if (q < 0 || q >= (int)ctx->qroute.size()) return {nullptr, -1};
  return {ctx->subs[ctx->qroute[q].first].plan, ctx->qroute[q].second};
}

// ------------------------------------------------------------------ join tree (GYO)
std::vector<std::string> shared_attrs(const lmfao_ctx *ctx, int a, int b) {
  std::vector<std::string> out;
  for (const Column &c : ctx->rels[a].cols)
    if (ctx->rels[b].col(c.attr) >= 0) out.push_back(c.attr);
  std::sort(out.begin(), out.end());
  return out;
}

// Parent links of a join tree by GYO ear removal: a relation whose attributes shared with
// the remaining relations all lie in one other remaining relation is an ear and hangs
// below it (the largest such relation). LMFAO_ERR_CYCLIC if the reduction stalls.
std::vector<int> gyo(const lmfao_ctx *ctx) {
  int n = (int)ctx->rels.size();
  std::vector<int> parent(n, -1);
  std::vector<bool> active(n, true);
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctx->rels[a].nrows < ctx->rels[b].nrows; });
  int left = n;
  while (left > 1) {
    bool found = false;
    for (int e : order) {
      if (!active[e]) continue;
      std::vector<std::string> sh;
      for (const Column &c : ctx->rels[e].cols) {
        for (int f = 0; f < n; ++f)
          if (f != e && active[f] && ctx->rels[f].col(c.attr) >= 0) { sh.push_back(c.attr); break; }
      }
      int best = -1;
      for (int f = 0; f < n; ++f) {
        if (f == e || !active[f]) continue;
        bool all = true;
        for (auto &a : sh) all = all && ctx->rels[f].col(a) >= 0;
        if (!all) continue;
        if (sh.empty() && best >= 0) continue;
        if (best < 0 || ctx->rels[f].nrows > ctx->rels[best].nrows) best = f;
      }
      if (best >= 0) {
        if (sh.empty()) throw Error(LMFAO_ERR_UNSUPPORTED, "the schema is disconnected (relation " +
                                                           ctx->rels[e].name + " shares no attribute)");
        parent[e] = best;
        active[e] = false;
        --left;
        found = true;
        break;
      }
    }
    if (!found) throw Error(LMFAO_ERR_CYCLIC, "the schema is cyclic: GYO reduction found no ear");
  }
  return parent;
}

JoinTree build_tree(const lmfao_ctx *ctx, const std::vector<int> &par_in, int root) {
  int n = (int)ctx->rels.size();
  // undirected adjacency, then re-root
  std::vector<std::vector<int>> adj(n);
  for (int i = 0; i < n; ++i)
    if (par_in[i] >= 0) { adj[i].push_back(par_in[i]); adj[par_in[i]].push_back(i); }
  JoinTree t;
  t.root = root;
  t.parent.assign(n, -1);
  t.children.assign(n, {});
  t.depth.assign(n, 0);
  std::vector<int> bfs{root};
  std::vector<bool> seen(n, false);
  seen[root] = true;
  for (size_t i = 0; i < bfs.size(); ++i) {
    int u = bfs[i];
    for (int v : adj[u])
      if (!seen[v]) {
        seen[v] = true;
        t.parent[v] = u;
        t.depth[v] = t.depth[u] + 1;
        t.children[u].push_back(v);
        bfs.push_back(v);
      }
  }
  if ((int)bfs.size() != n) throw Error(LMFAO_ERR_ARG, "join tree does not connect all relations");
  for (int i = n - 1; i >= 1; --i) t.post.push_back(bfs[i]);
  // running intersection: every attribute's relations form a connected subtree
  for (int r = 0; r < n; ++r)
    for (const Column &c : ctx->rels[r].cols) {
      int holders = 0, linked = 0;
      for (int s = 0; s < n; ++s)
        if (ctx->rels[s].col(c.attr) >= 0) {
          ++holders;
          if (t.parent[s] >= 0 && ctx->rels[t.parent[s]].col(c.attr) >= 0) ++linked;
        }
      if (holders - linked != 1)
        throw Error(LMFAO_ERR_ARG, "join tree violates the running intersection property on attribute " + c.attr);
    }
  return t;
}

// relation holding attribute a that is closest to the root of tree t (ties: lowest id)
int home_of(const lmfao_ctx *ctx, const JoinTree &t, const std::string &a) {
  int best = -1;
  for (int r = 0; r < (int)ctx->rels.size(); ++r)
    if (ctx->rels[r].col(a) >= 0 && (best < 0 || t.depth[r] < t.depth[best])) best = r;
  if (best < 0) throw Error(LMFAO_ERR_ARG, "unknown attribute " + a);
  return best;
}

// ------------------------------------------------------------------ logical plan (Section 2)
std::string term_name(const std::vector<FactorIn> &fs) {
  if (fs.empty()) return "1";
  std::vector<std::string> v;
  for (auto &f : fs) v.push_back(f.fn == LMFAO_FN_POW ? f.attr + "^" + std::to_string(f.param) : f.attr);
  std::sort(v.begin(), v.end());
  std::string s;
  for (auto &x : v) s += (s.empty() ? "" : "*") + x;
  return s;
}

LogicalPlan build_logical(const lmfao_ctx *ctx, const JoinTree &t, const int32_t *qroot) {
  int n = (int)ctx->rels.size();
  LogicalPlan L;
  std::vector<std::vector<int>> adj(n);
  for (int i = 0; i < n; ++i)
    if (t.parent[i] >= 0) { adj[i].push_back(t.parent[i]); adj[t.parent[i]].push_back(i); }
  std::map<std::tuple<int, int, std::vector<std::string>>, int> vmap;
  // per query: views toward its root
  for (int q = 0; q < (int)ctx->queries.size(); ++q) {
    const QueryIn &Q = ctx->queries[q];
    int rho = (qroot && qroot[q] >= 0) ? qroot[q] : -1;
    if (rho >= n) throw Error(LMFAO_ERR_ARG, "query root out of range");
    if (rho < 0) {  // heuristic: the relation holding the group-by attribute with the largest domain
      int64_t bestdom = -1;
      for (auto &g : Q.gb) {
        int h = home_of(ctx, t, g.attr);
        const Column &c = ctx->rels[h].cols[ctx->rels[h].col(g.attr)];
        int64_t dom = g.kind == LMFAO_GB_BUCKET ? (int64_t)g.thr.size() + 1 : c.domain;
        if (dom > bestdom) { bestdom = dom; rho = h; }
      }
      if (rho < 0) rho = t.root;
    }
    L.query_root.push_back(rho);
    // orient the tree toward rho
    std::vector<int> par(n, -1), bfs{rho};
    std::vector<bool> seen(n, false);
    seen[rho] = true;
    for (size_t i = 0; i < bfs.size(); ++i)
      for (int v : adj[bfs[i]])
        if (!seen[v]) { seen[v] = true; par[v] = bfs[i]; bfs.push_back(v); }
    std::vector<std::vector<int>> sub(n);  // subtree of u toward rho
    for (int i = n - 1; i >= 0; --i) {
      int u = bfs[i];
      sub[u].push_back(u);
      if (par[u] >= 0) sub[par[u]].insert(sub[par[u]].end(), sub[u].begin(), sub[u].end());
    }
    auto in_sub = [&](int u, const std::string &a) {
      for (int r : sub[u]) if (ctx->rels[r].col(a) >= 0) return true;
      return false;
    };
    std::vector<int> vid(n, -1);
    for (int i = n - 1; i >= 1; --i) {  // leaves first
      int u = bfs[i], v = par[u];
      std::set<std::string> key;
      for (auto &a : shared_attrs(ctx, u, v)) key.insert(a);
      for (auto &g : Q.gb) if (in_sub(u, g.attr)) key.insert(g.attr);
      std::vector<std::string> kv(key.begin(), key.end());
      auto k = std::make_tuple(u, v, kv);
      int id;
      auto it = vmap.find(k);
      if (it == vmap.end()) {
        id = (int)L.views.size();
        vmap[k] = id;
        LogicalView lv;
        lv.from = u; lv.to = v; lv.key = kv;
        L.views.push_back(lv);
      } else id = it->second;
      vid[u] = id;
      LogicalView &lv = L.views[id];
      lv.queries.insert(q);
      for (auto &agg : Q.aggs) {
        std::vector<FactorIn> part;
        for (auto &f : agg) if (in_sub(u, f.attr)) part.push_back(f);
        lv.aggs.insert(term_name(part));
      }
      for (int w : adj[u]) if (w != v && vid[w] >= 0) lv.deps.insert(vid[w]);
    }
    // the query depends on the views into rho
    (void)vid;
  }
  // groups by rounds: an item is computed at its node once all views it reads exist
  int nv = (int)L.views.size(), nq = (int)ctx->queries.size();
  std::vector<int> vgroup(nv, -1), qgroup(nq, -1);
  std::vector<std::set<int>> qdeps(nq);
  for (int v = 0; v < nv; ++v)
    for (int q : L.views[v].queries)
      if (L.views[v].to == L.query_root[q]) qdeps[q].insert(v);
  int done = 0;
  while (done < nv + nq) {
    std::map<int, LogicalGroup> round;
    for (int v = 0; v < nv; ++v) {
      if (vgroup[v] >= 0) continue;
      bool ok = true;
      for (int d : L.views[v].deps) ok = ok && vgroup[d] >= 0;
      if (ok) round[L.views[v].from].views.push_back(v);
    }
    for (int q = 0; q < nq; ++q) {
      if (qgroup[q] >= 0) continue;
      bool ok = true;
      for (int d : qdeps[q]) ok = ok && vgroup[d] >= 0;
      if (ok) round[L.query_root[q]].queries.push_back(q);
    }
    if (round.empty()) throw Error(LMFAO_ERR_ARG, "view dependencies do not resolve");
    // number groups: views toward the leaves-to-root order, stable by node id
    std::vector<std::pair<int, LogicalGroup>> items(round.begin(), round.end());
    for (auto &it : items) {
      LogicalGroup g = it.second;
      g.node = it.first;
      int gid = (int)L.groups.size();
      for (int v : g.views) for (int d : L.views[v].deps) g.deps.insert(vgroup[d]);
      for (int q : g.queries) for (int d : qdeps[q]) g.deps.insert(vgroup[d]);
      for (int v : g.views) { vgroup[v] = gid; ++done; }
      for (int q : g.queries) { qgroup[q] = gid; ++done; }
      L.groups.push_back(g);
    }
  }
  return L;
}

}  // namespace

// ======================================================================================
// physical planning
// ======================================================================================
namespace {

struct Planner {
  lmfao_ctx *ctx;
  PhysPlan &P;
  const JoinTree &t;
  cudaStream_t s;

  Planner(lmfao_ctx *c, PhysPlan &p, const JoinTree &tr) : ctx(c), P(p), t(tr), s(c->stream) {}

  const Relation &R(int r) const { return ctx->rels[r]; }

  int child_toward(int r, int h) const {  // child of r on the path to h (h in subtree(r), h != r)
    int x = h;
    while (t.parent[x] != r) {
      x = t.parent[x];
      if (x < 0) throw Error(LMFAO_ERR_ARG, "internal: relation not below");
    }
    return x;
  }
  int fac_id(const Fac &f) {
    auto it = P.facmap.find(f);
    if (it != P.facmap.end()) return it->second;
    int id = (int)P.facs.size();
    P.facs.push_back(f);
    P.facmap[f] = id;
    return id;
  }
  int gitem_id(const GroupItem &g) {
    auto it = P.gmap.find(g);
    if (it != P.gmap.end()) return it->second;
    int id = (int)P.gitems.size();
    P.gitems.push_back(g);
    P.gmap[g] = id;
    return id;
  }

  // ---- views
  void init_views() {
    int n = (int)ctx->rels.size();
    P.views.assign(n, View{});
    for (int r : t.post) {
      View &v = P.views[r];
      v.rel = r;
      v.parent = t.parent[r];
      for (auto &a : shared_attrs(ctx, r, v.parent)) {
        const Column &c = R(r).cols[R(r).col(a)];
        const Column &pc = R(v.parent).cols[R(v.parent).col(a)];
        if (c.role != LMFAO_KEY || pc.role != LMFAO_KEY || c.dtype != LMFAO_I32)
          throw Error(LMFAO_ERR_ARG, "join attribute " + a + " must be a KEY column in every relation");
        if (c.domain != pc.domain)
          throw Error(LMFAO_ERR_ARG, "join attribute " + a + " declares different domains");
        v.keycols.push_back(R(r).col(a));
        v.pkeycols.push_back(R(v.parent).col(a));
        v.keydom.push_back(c.domain);
      }
      if ((int)v.keycols.size() > MAXK) throw Error(LMFAO_ERR_UNSUPPORTED, "join key with more than 4 attributes");
      v.nkeys = 1;
      for (int64_t d : v.keydom) {
        v.nkeys *= d;
        if (v.nkeys > (int64_t(1) << 28))
          throw Error(LMFAO_ERR_UNSUPPORTED, "join key domain of " + R(r).name + " exceeds 2^28 cells");
      }
    }
    for (int r : t.post) view_col(r, {});  // COUNT columns
  }

  int view_col(int r, const Term &term) {
    View &v = P.views[r];
    auto it = v.colmap.find(term);
    if (it != v.colmap.end()) return it->second;
    ViewCol vc;
    std::map<int, Term> parts;
    for (int f : term) {
      const Fac &fc = P.facs[f];
      if (!fc.ind) vc.integral = false;
      if (fc.rel == r) vc.local.push_back(f);
      else parts[child_toward(r, fc.rel)].push_back(f);
    }
    for (int c : t.children[r]) {
      int cc = view_col(c, parts.count(c) ? parts[c] : Term{});
      vc.child.push_back({c, cc});
    }
    View &v2 = P.views[r];  // re-fetch (recursion does not resize, but keep it explicit)
    int id = (int)v2.cols.size();
    v2.cols.push_back(vc);
    v2.colmap[term] = id;
    return id;
  }

  int view_code(int r, int gid) {
    View &v = P.views[r];
    auto it = v.codemap.find(gid);
    if (it != v.codemap.end()) return it->second;
    CodeSpec cs;
    const GroupItem &g = P.gitems[gid];
    if (g.rel == r) cs.group = gid;
    else {
      cs.child_rel = child_toward(r, g.rel);
      cs.child_code = view_code(cs.child_rel, gid);
    }
    View &v2 = P.views[r];
    int id = (int)v2.codes.size();
    v2.codes.push_back(cs);
    v2.codemap[gid] = id;
    return id;
  }

  // ---- root level
  int rowslot(int col) {
    auto it = P.rowslot.find(col);
    if (it != P.rowslot.end()) return it->second;
    int id = (int)P.rowcols.size();
    if (id >= MAXRC) throw Error(LMFAO_ERR_UNSUPPORTED, "more than 24 root columns read per tuple");
    P.rowcols.push_back(col);
    P.rowslot[col] = id;
    return id;
  }
  int mono_id(std::vector<int> fs) {
    std::sort(fs.begin(), fs.end());
    auto it = P.monomap.find(fs);
    if (it != P.monomap.end()) return it->second;
    int id = (int)P.monos.size();
    P.monos.push_back(fs);
    P.monomap[fs] = id;
    return id;
  }
  int rt_id(int mono, const std::vector<std::pair<int, int>> &parts, bool integral) {
    auto k = std::make_pair(mono * 2 + (integral ? 1 : 0), parts);
    auto it = P.rtmap.find(k);
    if (it != P.rtmap.end()) return it->second;
    int id = (int)P.rts.size();
    P.rts.push_back({mono, parts, integral});
    P.rtmap[k] = id;
    return id;
  }
  int psi_id(std::vector<int> segf, const std::vector<std::pair<int, int>> &parts, bool integral) {
    std::sort(segf.begin(), segf.end());
    std::vector<int> key = segf;
    key.push_back(integral ? -2 : -1);
    auto k = std::make_pair(key, parts);
    auto it = P.psimap.find(k);
    if (it != P.psimap.end()) return it->second;
    int id = (int)P.psis.size();
    P.psis.push_back({segf, parts, integral});
    P.psimap[k] = id;
    return id;
  }

  int seg_digit_of(int col) const {
    for (size_t i = 0; i < P.segcols.size(); ++i) if (P.segcols[i] == col) return (int)i;
    return -1;
  }

  void choose_segments(const lmfao_plan_opts &o) {
    int root = t.root;
    int seg = -1;
    if (o.planner == LMFAO_PLAN_FORCED && o.segment_rel != -2) {
      seg = o.segment_rel;
      if (seg >= 0 && t.parent[seg] != root)
        throw Error(LMFAO_ERR_ARG, "segment relation must be a child of the root relation");
    } else {
      int64_t best = 0;
      int64_t cap = std::max<int64_t>(1, R(root).nrows / 4);
      for (int c : t.children[root]) {
        const View &v = P.views[c];
        if (v.nkeys > best && v.nkeys <= cap && v.nkeys <= (int64_t(1) << 26)) { best = v.nkeys; seg = c; }
      }
    }
    P.segrel = seg;
    P.nseg = 1;
    P.prefix_len = 0;
    if (seg >= 0) {
      const View &v = P.views[seg];
      P.segcols = v.pkeycols;
      P.segdom = v.keydom;
      for (int64_t d : P.segdom) P.nseg *= d;
      if (P.segcols.size() > 8) throw Error(LMFAO_ERR_UNSUPPORTED, "segment key with more than 8 attributes");
      // Trie order of the segment key: the key of the outer child with the largest subtree
      // whose key is a proper part of the segment key goes first, so that its view is
      // constant over contiguous blocks of segments (the prefix).
      int best = -1, bestw = -1;
      for (int c : t.children[root]) {
        if (c == seg) continue;
        const View &cv = P.views[c];
        bool inside = !cv.pkeycols.empty() && cv.pkeycols.size() < P.segcols.size();
        for (int pc : cv.pkeycols)
          inside = inside && std::find(P.segcols.begin(), P.segcols.end(), pc) != P.segcols.end();
        if (!inside) continue;
        int width = 0;
        std::vector<int> st{c};
        while (!st.empty()) {
          int x = st.back();
          st.pop_back();
          width += (int)R(x).cols.size();
          for (int y : t.children[x]) st.push_back(y);
        }
        if (width > bestw) { bestw = width; best = c; }
      }
      if (best >= 0) {
        std::vector<int> cols, rest;
        std::vector<int64_t> dom, rdom;
        const View &bv = P.views[best];
        for (size_t i = 0; i < P.segcols.size(); ++i) {
          bool in = std::find(bv.pkeycols.begin(), bv.pkeycols.end(), P.segcols[i]) != bv.pkeycols.end();
          (in ? cols : rest).push_back(P.segcols[i]);
          (in ? dom : rdom).push_back(P.segdom[i]);
        }
        P.prefix_len = (int)cols.size();
        cols.insert(cols.end(), rest.begin(), rest.end());
        dom.insert(dom.end(), rdom.begin(), rdom.end());
        P.segcols = cols;
        P.segdom = dom;
      }
    }
    P.kind.assign(ctx->rels.size(), 0);
    P.branch.assign(ctx->rels.size(), -1);
    for (int c : t.children[root]) {
      bool outer = seg >= 0;
      for (int pc : P.views[c].pkeycols) outer = outer && seg_digit_of(pc) >= 0;
      (outer ? P.outer : P.inner).push_back(c);
    }
    if (P.outer.size() > MAXOUT || P.inner.size() > MAXIN)
      throw Error(LMFAO_ERR_UNSUPPORTED, "too many children of the root relation");
    for (int r = 0; r < (int)ctx->rels.size(); ++r) {
      if (r == root) continue;
      int b = r;
      while (t.parent[b] != root) b = t.parent[b];
      P.branch[r] = b;
      P.kind[r] = std::find(P.outer.begin(), P.outer.end(), b) != P.outer.end() ? 1 : 2;
    }
  }

  int outer_idx(int c) const { return (int)(std::find(P.outer.begin(), P.outer.end(), c) - P.outer.begin()); }
  int inner_idx(int c) const { return (int)(std::find(P.inner.begin(), P.inner.end(), c) - P.inner.begin()); }

  Fac make_fac(const std::string &attr, bool ind, int pow, int op, float tv) {
    int h = home_of(ctx, t, attr);
    Fac f;
    f.rel = h;
    f.col = R(h).col(attr);
    f.ind = ind ? 1 : 0;
    f.pow = ind ? 1 : pow;
    f.op = ind ? op : 0;
    f.t = ind ? tv : 0.f;
    return f;
  }

  DGroupRef group_ref(int gid, int64_t stride) {
    const GroupItem &g = P.gitems[gid];
    DGroupRef r{};
    r.stride = stride;
    r.kind = g.kind;
    r.thr0 = (int)P.thr.size();
    r.nthr = (int)g.thr.size();
    P.thr.insert(P.thr.end(), g.thr.begin(), g.thr.end());
    if (g.rel == t.root) {
      int d = seg_digit_of(g.col);
      if (d >= 0 && g.kind == LMFAO_GB_VALUE) { r.src = 0; r.a = d; }
      else { r.src = 2; r.a = rowslot(g.col); }
    } else {
      int b = P.branch[g.rel];
      int code = view_code(b, gid);
      if (P.kind[g.rel] == 1) { r.src = 1; r.a = outer_idx(b); r.b = code; }
      else { r.src = 3; r.a = inner_idx(b); r.b = code; }
    }
    return r;
  }

  // One output item: aggregate a of query q (a = -1: the query's COUNT(*)), split into
  // its outer part psi (segment level), its row factors, its inner view columns and its
  // outer / inner group references.
  struct ItemD {
    int q = 0, a = 0;
    bool integral = true;
    int psi = 0;
    std::vector<int> rowf;
    std::vector<std::pair<int, int>> ipart;
    std::vector<DGroupRef> og, ig;
    int64_t out = 0, cellmul = 1;
    bool outer_dep = false;
    int leaf = -1;  // filter index within the filter family (-1: filter kept as indicators)
  };

  // Filter family: the distinct filters of the batch when they are pairwise disjoint
  // conjunctions (the leaves of a decision-tree level). Each tuple satisfies at most one;
  // its index is computed once per tuple instead of evaluating every filtered item.
  struct Family {
    std::vector<std::vector<int>> filters;  // predicate factor ids per filter
    std::vector<int> preds;                 // distinct predicate factor ids
    std::vector<int> qfilter;               // per query: filter index or -1
  } fam;
  bool use_family = false;

  static bool complementary(const Fac &a, const Fac &b) {
    if (a.rel != b.rel || a.col != b.col || a.t != b.t) return false;
    auto pairs = [&](int x, int y) { return (a.op == x && b.op == y) || (a.op == y && b.op == x); };
    return pairs(LMFAO_LE, LMFAO_GT) || pairs(LMFAO_LT, LMFAO_GE) || pairs(LMFAO_EQ, LMFAO_NE);
  }

  bool detect_family() {
    fam = Family{};
    fam.qfilter.assign(ctx->queries.size(), -1);
    for (int q = 0; q < (int)ctx->queries.size(); ++q) {
      const QueryIn &Q = ctx->queries[q];
      if (Q.filters.empty()) continue;
      std::vector<int> f;
      for (auto &pd : Q.filters) f.push_back(fac_id(make_fac(pd.attr, true, 1, pd.op, pd.t)));
      std::sort(f.begin(), f.end());
      f.erase(std::unique(f.begin(), f.end()), f.end());
      int at = -1;
      for (size_t i = 0; i < fam.filters.size(); ++i) if (fam.filters[i] == f) at = (int)i;
      if (at < 0) { fam.filters.push_back(f); at = (int)fam.filters.size() - 1; }
      fam.qfilter[q] = at;
    }
    const int K = (int)fam.filters.size();
    if (K < 2 || K > FMAXFAM) return false;
    for (int a = 0; a < K; ++a)
      for (int b = a + 1; b < K; ++b) {
        bool disjoint = false;
        for (int x : fam.filters[a])
          for (int y : fam.filters[b]) disjoint = disjoint || complementary(P.facs[x], P.facs[y]);
        if (!disjoint) return false;
      }
    std::set<int> ps;
    for (auto &f : fam.filters) ps.insert(f.begin(), f.end());
    fam.preds.assign(ps.begin(), ps.end());
    if ((int)fam.preds.size() > FMAXBIT) return false;
    for (int pfac : fam.preds) {
      const Fac &fc = P.facs[pfac];
      if (fc.rel == t.root) {
        if (seg_digit_of(fc.col) >= 0) return false;  // predicates on segment-key digits stay indicators
        continue;
      }
      // a predicate on a non-root relation is one bit of its (unique) joined tuple
      if (P.views[P.branch[fc.rel]].count_bound > 1.0) return false;
    }
    return true;
  }

  std::vector<ItemD> decompose() {
    int root = t.root;
    int64_t fo = 0, io = 0;
    std::vector<ItemD> items;
    for (int q = 0; q < (int)ctx->queries.size(); ++q) {
      const QueryIn &Q = ctx->queries[q];
      QueryOut qo;
      qo.naggs = (int)Q.aggs.size();
      if ((int)Q.gb.size() > MAXGR) throw Error(LMFAO_ERR_UNSUPPORTED, "more than 4 group-by attributes");
      for (auto &g : Q.gb) {
        int h = home_of(ctx, t, g.attr);
        const Column &c = R(h).cols[R(h).col(g.attr)];
        GroupItem gi;
        gi.rel = h;
        gi.col = R(h).col(g.attr);
        gi.kind = g.kind;
        if (g.kind == LMFAO_GB_VALUE) {
          if (c.role == LMFAO_CONT) throw Error(LMFAO_ERR_ARG, "VALUE group-by on continuous attribute " + g.attr);
          gi.dom = c.domain;
        } else {
          gi.thr = g.thr;
          gi.dom = (int64_t)g.thr.size() + 1;
        }
        qo.gitems.push_back(gitem_id(gi));
        qo.dom.push_back(gi.dom);
        qo.cells *= gi.dom;
        if (qo.cells > (int64_t(1) << 28)) throw Error(LMFAO_ERR_UNSUPPORTED, "group-by domain exceeds 2^28 cells");
      }
      qo.fo = fo;
      qo.io = io;
      fo += qo.cells * qo.naggs;
      io += qo.cells * (1 + qo.naggs);
      std::vector<int64_t> stride(qo.dom.size(), 1);
      for (int i = (int)qo.dom.size() - 2; i >= 0; --i) stride[i] = stride[i + 1] * qo.dom[i + 1];
      std::vector<int> inds;
      const int leaf = use_family ? fam.qfilter[q] : -1;
      if (leaf < 0)
        for (auto &p : Q.filters) inds.push_back(fac_id(make_fac(p.attr, true, 1, p.op, p.t)));
      for (int a = -1; a < qo.naggs; ++a) {
        ItemD it;
        it.q = q;
        it.a = a;
        it.leaf = leaf;
        Term term = inds;
        if (a >= 0)
          for (auto &f : Q.aggs[a]) {
            term.push_back(fac_id(make_fac(f.attr, false, f.fn == LMFAO_FN_POW ? f.param : 1, 0, 0.f)));
            it.integral = false;
          }
        if (a >= 0) qo.integral.push_back(it.integral ? 1 : 0);
        std::sort(term.begin(), term.end());
        // split the product by where its factors live
        std::vector<int> segf;
        std::map<int, Term> bparts;
        for (int f : term) {
          const Fac &fc = P.facs[f];
          if (fc.rel == root) {
            int d = seg_digit_of(fc.col);
            if (d >= 0) segf.push_back(f);
            else { rowslot(fc.col); it.rowf.push_back(f); }
          } else bparts[P.branch[fc.rel]].push_back(f);
        }
        std::vector<std::pair<int, int>> opart;
        it.outer_dep = !segf.empty();
        for (int c : P.outer) {
          int col = view_col(c, bparts.count(c) ? bparts[c] : Term{});
          opart.push_back({outer_idx(c), col});
          if (col != 0) it.outer_dep = true;
        }
        for (int c : P.inner) {
          int col = view_col(c, bparts.count(c) ? bparts[c] : Term{});
          it.ipart.push_back({inner_idx(c), col});
        }
        it.psi = psi_id(segf, opart, it.integral);
        for (size_t i = 0; i < qo.gitems.size(); ++i) {
          DGroupRef g = group_ref(qo.gitems[i], stride[i]);
          (g.src <= 1 ? it.og : it.ig).push_back(g);
        }
        if (!it.og.empty()) it.outer_dep = true;
        it.out = it.integral ? qo.io + 1 + a : qo.fo + a;
        it.cellmul = it.integral ? 1 + qo.naggs : qo.naggs;
        items.push_back(it);
      }
      P.qout.push_back(qo);
    }
    P.nfsum = fo;
    P.nicnt = io;
    return items;
  }

  int add_grefs(const std::vector<DGroupRef> &g) {
    int at = (int)P.grefs.size();
    P.grefs.insert(P.grefs.end(), g.begin(), g.end());
    return at;
  }

  // Generic routing: per-segment sums (B0) where the item has no inner group, per-tuple
  // accumulation (B2) otherwise.
  void route_generic(const std::vector<ItemD> &items, int mode) {
    for (const ItemD &it : items) {
      int rt = rt_id(mono_id(it.rowf), it.ipart, it.integral);
      bool b0 = it.ig.empty() && mode != LMFAO_MODE_PER_TUPLE;
      if (b0) {
        auto &lst = it.integral ? P.b0i : P.b0f;
        int pos = (int)(std::find(lst.begin(), lst.end(), rt) - lst.begin());
        int cap = it.integral ? NI0_MAX : NB0_MAX;
        if (pos == (int)lst.size()) {
          if ((int)lst.size() >= cap) b0 = false;
          else lst.push_back(rt);
        }
        if (b0) {
          DCombItem c{};
          c.sel = -1;
          c.psi = it.psi;
          c.block = -1;
          c.col = pos;
          c.integral = it.integral;
          c.og0 = add_grefs(it.og);
          c.nog = (int)it.og.size();
          c.out = it.out;
          c.cellmul = it.cellmul;
          P.comb.push_back(c);
        }
      }
      if (!b0) {
        DB2Item c{};
        c.psi = it.psi;
        c.rterm = rt;
        c.integral = it.integral;
        c.og0 = add_grefs(it.og);
        c.nog = (int)it.og.size();
        c.ig0 = add_grefs(it.ig);
        c.nig = (int)it.ig.size();
        c.out = it.out;
        c.cellmul = it.cellmul;
        P.b2.push_back(c);
      }
    }
  }

  // Routing of the specialised root pass (at most one inner child): B0 as the outer product
  // of monomials and inner view columns, B1 per-segment group histograms, B3 partial view
  // from the root to the inner relation. Returns false when the batch needs the generic pass.
  // Records why the specialised root pass does not take the batch (reported by the plan's
  // description) and declines.
  bool decline(const char *why) {
    P.fast_why += std::string(P.fast_why.empty() ? "" : "; ") + (use_family ? "as a filter family: " : "") + why;
    return false;
  }

  bool route_fast(const std::vector<ItemD> &items) {
    if (P.inner.size() > 1) return decline("P.inner.size() > 1");
    if (P.inner.size() == 1) {
      const View &v = P.views[P.inner[0]];
      if (v.keycols.size() > 2) return decline("v.keycols.size() > 2");
      if (v.count_bound * 4096.0 >= 16777216.0) return decline("v.count_bound * 4096.0 >= 16777216.0");  // exact integral sums in FP32
    }
    auto &F = P.fast;
    F = PhysPlan::Fast{};
    F.wcols.push_back(0);
    auto mono_of = [&](std::vector<int> fs) -> int {
      std::sort(fs.begin(), fs.end());
      for (size_t j = 0; j < F.monos.size(); ++j) if (F.monos[j] == fs) return (int)j;
      F.monos.push_back(fs);
      return (int)F.monos.size() - 1;
    };
    auto wcol_of = [&](int c) -> int {
      for (size_t w = 0; w < F.wcols.size(); ++w) if (F.wcols[w] == c) return (int)w;
      F.wcols.push_back(c);
      return (int)F.wcols.size() - 1;
    };
    struct Pending { ItemD it; int j, w; int kind; int set; };
    std::vector<Pending> pend;
    F.b3leaf = 1;
    bool b3_plain = false, b3_leafed = false;
    const int K = use_family ? (int)fam.filters.size() : 0;
    // Items of a filter family grouped by inner codes go to the leaf-split view from the root
    // to the inner relation (inner keys x leaves x columns; its float part in global memory
    // when it does not fit a CTA), or with LMFAO_LEAF_ITEMS=cta to per-CTA (leaf, code) cells:
    // one shared atomic per item and tuple instead of per column, which measured slower on
    // the decision-tree level (5.5 ms against 3.3 ms at 84M tuples).
    bool leaf_items_cta = false;
    if (K > 1 && P.inner.size() == 1)
      if (const char *e = std::getenv("LMFAO_LEAF_ITEMS")) leaf_items_cta = std::string(e) == "cta";
    for (const ItemD &it : items) {
      int j = mono_of(it.rowf);
      int vcol = it.ipart.empty() ? 0 : it.ipart[0].second;
      bool all_view = true, all_row = true;
      for (auto &g : it.ig) {
        all_view = all_view && g.src == 3;
        all_row = all_row && g.src == 2;
      }
      if (it.leaf >= 0) {
        if (!it.ig.empty() && all_view && !it.outer_dep && !it.ipart.empty() && !leaf_items_cta) {
          b3_leafed = true;
          pend.push_back({it, j, vcol, 3, -1});
        } else if (!it.ig.empty() && (all_row || (all_view && leaf_items_cta)) && !it.outer_dep) {
          pend.push_back({it, j, wcol_of(vcol), 4, -1});
        } else {
          if (it.ig.size() > 1) return decline("it.ig.size() > 1");
          // per-segment sums grouped by the tuple's filter index (and at most one inner code)
          DGroupRef lr{};
          lr.src = 4;
          std::vector<DGroupRef> key{lr};
          key.insert(key.end(), it.ig.begin(), it.ig.end());
          std::vector<int64_t> dom{K};
          int64_t G = K;
          for (size_t i = 1; i < key.size(); ++i) {
            const DGroupRef &g = key[i];
            int64_t dd = g.src == 3 ? P.gitems[code_group(P.inner[0], g.b)].dom
                                    : (g.kind == LMFAO_GB_BUCKET ? g.nthr + 1 : gdom_of_slot(g));
            dom.push_back(dd);
            G *= dd;
          }
          if (G > 4096) return decline("G > 4096");
          int set = find_or_add_b1(key, dom, G);
          if (set < 0) return decline("set < 0");
          ItemD it2 = it;
          it2.ig = key;
          it2.ig[0].stride = 0;  // the filter index selects; it is not an output group
          pend.push_back({it2, j, wcol_of(vcol), 1, set});
        }
        continue;
      }
      // Items that do not depend on the outer side and read inner view columns (or group by
      // inner codes) go to the view from the root to the inner relation (B3); the rest of the
      // ungrouped items are per-segment sums (B0).
      if (!it.outer_dep && all_view && !it.ipart.empty() && (vcol != 0 || !it.ig.empty())) {
        b3_plain = true;
        pend.push_back({it, j, vcol, 3, -1});
        continue;
      }
      if (it.ig.empty()) {
        pend.push_back({it, j, wcol_of(vcol), 0, -1});
        continue;
      }
      if (it.ig.size() > 2) return decline("it.ig.size() > 2");
      // B1 set keyed by its group references (without the query strides)
      std::vector<DGroupRef> key = it.ig;
      int64_t G = 1;
      std::vector<int64_t> dom;
      for (auto &g : key) {
        int64_t d = g.src == 3 ? P.gitems[code_group(P.inner[0], g.b)].dom
                               : (g.kind == LMFAO_GB_BUCKET ? g.nthr + 1 : gdom_of_slot(g));
        dom.push_back(d);
        G *= d;
      }
      if (G > 4096) return decline("G > 4096");
      int set = find_or_add_b1(key, dom, G);
      if (set < 0) return decline("set < 0");
      pend.push_back({it, j, wcol_of(vcol), 1, set});
    }
    if (b3_plain && b3_leafed) return decline("b3_plain && b3_leafed");
    if (b3_leafed) F.b3leaf = K;
    // Lean variant: root-level monomials of degree <= 2 over at most 3 value columns and no
    // indicators. The monomial list becomes the full basis (1, x_i, x_i x_j) in the order
    // the kernel computes it.
    F.lean = false;
    {
      bool ok = P.inner.size() <= 1 && (P.inner.empty() || P.views[P.inner[0]].keycols.size() == 1) && !use_family;
      std::vector<int> xcols;
      std::vector<std::map<int, int>> exps(F.monos.size());
      for (size_t j = 0; j < F.monos.size() && ok; ++j) {
        int deg = 0;
        for (int f : F.monos[j]) {
          const Fac &fc = P.facs[f];
          if (fc.ind) { ok = false; break; }
          if (std::find(xcols.begin(), xcols.end(), fc.col) == xcols.end()) xcols.push_back(fc.col);
          exps[j][fc.col] += fc.pow;
          deg += fc.pow;
        }
        if (deg > 2) ok = false;
      }
      if (ok && xcols.size() <= 3) {
        std::vector<std::map<int, int>> basis{{}};
        for (int c : xcols) basis.push_back({{c, 1}});
        for (size_t a = 0; a < xcols.size(); ++a)
          for (size_t b = a; b < xcols.size(); ++b) {
            std::map<int, int> e;
            e[xcols[a]] += 1;
            e[xcols[b]] += 1;
            basis.push_back(e);
          }
        std::vector<int> remap(F.monos.size());
        for (size_t j = 0; j < F.monos.size(); ++j)
          remap[j] = (int)(std::find(basis.begin(), basis.end(), exps[j]) - basis.begin());
        std::vector<std::vector<int>> bm;
        for (auto &e : basis) {
          std::vector<int> fs;
          for (int c : xcols)  // first-order factors first so the kernel's column order is xcols
            for (int q = 0; q < (e.count(c) ? e.at(c) : 0); ++q) {
              Fac f;
              f.rel = t.root;
              f.col = c;
              fs.push_back(fac_id(f));
            }
          bm.push_back(fs);
        }
        F.monos = bm;
        for (auto &pd : pend) pd.j = remap[pd.j];
        F.lean = true;
        F.lean_cols = xcols;
      }
    }
    if (F.monos.size() > FMAXM || F.wcols.size() > FMAXW) return decline("F.monos.size() > FMAXM || F.wcols.size() > FMAXW");
    if (!F.lean && !fast_shape_ok((int)F.monos.size(), (int)F.wcols.size())) return decline("!F.lean && !fast_shape_ok((int)F.monos.size(), (int)F.wcols.size())");
    int nfac = 0;
    std::set<int> xcols;
    for (auto &m : F.monos)
      for (int f : m) {
        if (P.facs[f].ind) ++nfac;
        else xcols.insert(P.facs[f].col);
      }
    if (nfac > FMAXF || (int)xcols.size() > FMAXX) return decline("nfac > FMAXF || (int)xcols.size() > FMAXX");
    if (P.inner.size() == 1 && P.views[P.inner[0]].nkeys * (int64_t)F.wcols.size() >= (int64_t(1) << 31)) return decline("P.inner.size() == 1 && P.views[P.inner[0]].nkeys * (int64_t)F.wcols.size() >= (int64_t(1) ");
    const int nw = (int)F.wcols.size();
    for (auto &pd : pend) {
      const ItemD &it = pd.it;
      if (pd.kind == 0) {
        DCombItem c{};
          c.sel = -1;
        c.psi = it.psi;
        c.block = -1;
        c.integral = it.integral;
        if (it.integral) {
          int pos = -1;
          for (size_t i = 0; i < F.int0.size(); ++i)
            if (F.int0[i].first == pd.j && F.int0[i].second == pd.w) pos = (int)i;
          if (pos < 0) {
            if ((int)F.int0.size() >= NI0_MAX) return decline("(int)F.int0.size() >= NI0_MAX");
            F.int0.push_back({pd.j, pd.w});
            pos = (int)F.int0.size() - 1;
          }
          c.col = pos;
        } else {
          c.col = pd.j * nw + pd.w;
        }
        c.og0 = add_grefs(it.og);
        c.nog = (int)it.og.size();
        c.out = it.out;
        c.cellmul = it.cellmul;
        P.comb.push_back(c);
      } else if (pd.kind == 1) {
        auto &S = F.b1[pd.set];
        // the column kind follows the column (an inner COUNT is integral even when the
        // outer factor of the item is not)
        bool mono_int = true;
        for (int f : F.monos[pd.j]) mono_int = mono_int && P.facs[f].ind;
        // with no inner child the tuple's view row is the constant COUNT 1 (integral)
        const bool colint =
            mono_int && (P.inner.empty() ? F.wcols[pd.w] == 0 : P.views[P.inner[0]].cols[F.wcols[pd.w]].integral);
        auto &cols = colint ? S.icols : S.fcols;
        int pos = -1;
        for (size_t i = 0; i < cols.size(); ++i) if (cols[i].first == pd.j && cols[i].second == pd.w) pos = (int)i;
        if (pos < 0) {
          if ((int)cols.size() >= FMAXC) return decline("(int)cols.size() >= FMAXC");
          cols.push_back({pd.j, pd.w});
          pos = (int)cols.size() - 1;
        }
        DCombItem c{};
          c.sel = -1;
        c.psi = it.psi;
        c.block = pd.set;
        c.integral = it.integral;
        c.yint = colint ? 1 : 0;
        c.sel = it.leaf;
        c.col = pos;
        c.og0 = add_grefs(it.og);
        c.nog = (int)it.og.size();
        c.ig0 = add_grefs(it.ig);
        c.nig = (int)it.ig.size();
        c.out = it.out;
        c.cellmul = it.cellmul;
        P.comb.push_back(c);
      } else if (pd.kind == 4) {
        PhysPlan::Fast::B4 b;
        b.j = pd.j;
        b.w = pd.w;
        b.integral = it.integral;
        b.sel = it.leaf;
        b.refs = it.ig;
        b.q = it.q;
        b.out = it.out;
        b.cellmul = it.cellmul;
        F.b4.push_back(b);
        if ((int)F.b4.size() > FMAXB4) return decline("(int)F.b4.size() > FMAXB4");
      } else {
        // the partial w_s * u_j is an exact integer when the monomial has only indicator
        // factors (or none): one integral column then serves integral and float items
        bool mono_int = true;
        for (int f : F.monos[pd.j]) mono_int = mono_int && P.facs[f].ind;
        if (it.integral && !mono_int) return decline("it.integral && !mono_int");
        int pos = -1;
        for (size_t i = 0; i < F.p3.size(); ++i) if (F.p3[i].first == pd.j && F.p3[i].second == mono_int) pos = (int)i;
        if (pos < 0) {
          if ((int)F.p3.size() >= FMAXC) return decline("(int)F.p3.size() >= FMAXC");
          F.p3.push_back({pd.j, mono_int});
          pos = (int)F.p3.size() - 1;
        }
        DB3Item b{};
        b.pint = mono_int ? 1 : 0;
        const View &v = P.views[P.inner[0]];
        b.w = it.integral ? pd.w : pd.w;  // FP64 view column; integral values are exact there
        (void)v;
        b.c = pos;
        b.leaf = it.leaf;
        b.integral = it.integral;
        b.ig0 = add_grefs(it.ig);
        b.nig = (int)it.ig.size();
        b.out = it.out;
        b.cellmul = it.cellmul;
        F.b3.push_back(b);
      }
    }
    if (use_family) {
      F.fam_k = K;
      F.fmask.assign(K, 0u);
      F.obits.clear();
      F.ibits.clear();
      F.rbits.clear();
      for (size_t pi = 0; pi < fam.preds.size(); ++pi) {
        const int pf = fam.preds[pi];
        const Fac &fc = P.facs[pf];
        for (int f = 0; f < K; ++f)
          if (std::find(fam.filters[f].begin(), fam.filters[f].end(), pf) != fam.filters[f].end())
            F.fmask[f] |= 1u << pi;
        if (fc.rel == t.root) {
          F.rbits.push_back({rowslot(fc.col), (int)pi, pf});
        } else {
          const int b = P.branch[fc.rel];
          const int col = view_col(b, Term{pf});  // filtered COUNT: 1 when the tuple satisfies it
          if (P.kind[fc.rel] == 1) F.obits.push_back({outer_idx(b), col, (int)pi});
          else F.ibits.push_back({col, (int)pi, 0});
        }
      }
    }
    if (F.lean) {
      for (auto &S : F.b1)
        if (S.refs.size() != 1 || S.refs[0].src != 3 || !S.fcols.empty() || S.icols.size() != 1 ||
            S.icols[0].first != 0 || S.icols[0].second != 0)
          F.lean = false;
      for (auto &c : F.p3)
        if (c.second && c.first != 0) F.lean = false;
      if (!F.lean && !fast_shape_ok((int)F.monos.size(), (int)F.wcols.size())) return decline("!F.lean && !fast_shape_ok((int)F.monos.size(), (int)F.wcols.size())");
    }
    F.on = true;
    return true;
  }

  int find_or_add_b1(const std::vector<DGroupRef> &key, const std::vector<int64_t> &dom, int64_t G) {
    auto &F = P.fast;
    for (size_t s2 = 0; s2 < F.b1.size(); ++s2) {
      auto &S = F.b1[s2];
      if (S.refs.size() != key.size()) continue;
      bool same = true;
      for (size_t i = 0; i < key.size(); ++i)
        same = same && S.refs[i].src == key[i].src && S.refs[i].a == key[i].a && S.refs[i].b == key[i].b &&
               S.refs[i].kind == key[i].kind && S.thrs[i] == thr_of(key[i]);
      if (same) return (int)s2;
    }
    if (F.b1.size() >= FMAXB1) return -1;
    PhysPlan::Fast::B1 S;
    S.refs = key;
    for (auto &g : key) S.thrs.push_back(thr_of(g));
    S.dom = dom;
    S.G = G;
    F.b1.push_back(S);
    return (int)F.b1.size() - 1;
  }

  int code_group(int r, int code) const {  // group item behind a view code
    const CodeSpec &cs = P.views[r].codes[code];
    if (cs.group >= 0) return cs.group;
    return code_group(cs.child_rel, cs.child_code);
  }
  std::vector<float> thr_of(const DGroupRef &g) const {
    return std::vector<float>(P.thr.begin() + g.thr0, P.thr.begin() + g.thr0 + g.nthr);
  }
  int64_t gdom_of_slot(const DGroupRef &g) const {  // VALUE code on a root column
    int col = P.rowcols[g.a];
    return R(t.root).cols[col].domain;
  }
};

}  // namespace

// ======================================================================================
// device-side setup of a plan
// ======================================================================================
namespace {

DViewRef view_ref(const View &v) {
  DViewRef r{};
  r.v64 = v.v64;
  r.v32 = v.v32;
  r.vint = v.vint;
  r.codes = v.vcodes;
  r.ncols = (int)v.cols.size();
  r.nint = v.nint;
  r.ncodes = (int)v.codes.size();
  r.nk = (int)v.keycols.size();
  int64_t st = 1;
  for (int i = r.nk - 1; i >= 0; --i) { r.kstride[i] = st; st *= v.keydom[i]; }
  return r;
}

DCol dcol(const Column &c) { return DCol{c.dev, c.dtype}; }

// Largest number of tuples per join-key value of every non-root relation, and an upper
// bound of each view's COUNT column (the product of multiplicities down the subtree).
void compute_multiplicities(lmfao_ctx *ctx, PhysPlan &P, const JoinTree &t) {
  cudaStream_t s = ctx->stream;
  for (int r : t.post) {
    View &v = P.views[r];
    std::vector<DCol> kc;
    std::vector<int64_t> st(v.keycols.size());
    int64_t acc = 1;
    for (int i = (int)v.keycols.size() - 1; i >= 0; --i) { st[i] = acc; acc *= v.keydom[i]; }
    for (int c : v.keycols) kc.push_back(dcol(ctx->rels[r].cols[c]));
    unsigned int *hist = (unsigned int *)P.arena.alloc(v.nkeys * 4 + 16);
    unsigned int *mx = hist + v.nkeys;
    int64_t *std_ = P.arena.upload(st, s);
    LMFAO_CUDA(cudaMemsetAsync(hist, 0, v.nkeys * 4 + 16, s));
    launch_key_multiplicity(kc.data(), (int)kc.size(), std_, ctx->rels[r].nrows, hist, s);
    launch_max_u32(hist, v.nkeys, mx, s);
    unsigned int h = 0;
    LMFAO_CUDA(cudaMemcpyAsync(&h, mx, 4, cudaMemcpyDeviceToHost, s));
    LMFAO_CUDA(cudaStreamSynchronize(s));
    v.maxmult = h;
    v.unique_keys = h <= 1;

    double b = std::max(1u, h);
    for (int c : t.children[r]) b *= P.views[c].count_bound;
    v.count_bound = b;
  }
}

void setup_views(lmfao_ctx *ctx, PhysPlan &P, const JoinTree &t, bool need32) {
  cudaStream_t s = ctx->stream;
  for (int r : t.post) {
    View &v = P.views[r];
    // integral column map
    v.intcol.assign(v.cols.size(), -1);
    std::vector<int> ic;
    for (size_t j = 0; j < v.cols.size(); ++j)
      if (v.cols[j].integral) { v.intcol[j] = (int)ic.size(); ic.push_back((int)j); }
    v.nint = (int)ic.size();
    size_t ncols = v.cols.size();
    v.v64 = (double *)P.arena.alloc(v.nkeys * ncols * 8);
    if (need32) v.v32 = (float *)P.arena.alloc(v.nkeys * ncols * 4);
    v.vint = (uint32_t *)P.arena.alloc(v.nkeys * std::max<size_t>(1, ic.size()) * 4);
    v.vcodes = (int32_t *)P.arena.alloc(v.nkeys * std::max<size_t>(1, v.codes.size()) * 4);
    int *icd = P.arena.upload(ic, s);
    // kernel descriptor
    DViewKernel d{};
    const Relation &Rr = ctx->rels[r];
    d.nrows = Rr.nrows;
    std::map<int, int> slot;
    auto sl = [&](int col) {
      auto it = slot.find(col);
      if (it != slot.end()) return it->second;
      int id = (int)slot.size();
      if (id >= MAXRC) throw Error(LMFAO_ERR_UNSUPPORTED, "view kernel reads more than 24 columns");
      slot[col] = id;
      d.in[id] = dcol(Rr.cols[col]);
      return id;
    };
    d.nk = (int)v.keycols.size();
    {
      int64_t st = 1;
      for (int i = d.nk - 1; i >= 0; --i) { d.kstride[i] = st; st *= v.keydom[i]; }
      for (int i = 0; i < d.nk; ++i) d.kcol[i] = sl(v.keycols[i]);
    }
    d.nchild = (int)t.children[r].size();
    if (d.nchild > MAXCH) throw Error(LMFAO_ERR_UNSUPPORTED, "relation with more than 8 children");
    for (int ci = 0; ci < d.nchild; ++ci) {
      const View &cv = P.views[t.children[r][ci]];
      d.child[ci] = view_ref(cv);
      for (int i = 0; i < d.child[ci].nk; ++i) d.child[ci].kcol[i] = sl(cv.pkeycols[i]);
    }
    std::vector<int> cfo{0}, cpo{0};
    std::vector<DFac> facs;
    std::vector<int2> parts;
    for (auto &vc : v.cols) {
      for (int f : vc.local) {
        const Fac &fc = P.facs[f];
        facs.push_back(DFac{sl(fc.col), fc.ind, fc.pow, fc.op, fc.t});
      }
      cfo.push_back((int)facs.size());
      for (auto &pc : vc.child) {
        int ci = (int)(std::find(t.children[r].begin(), t.children[r].end(), pc.first) - t.children[r].begin());
        parts.push_back(make_int2(ci, pc.second));
      }
      cpo.push_back((int)parts.size());
    }
    std::vector<int4> cdesc;
    std::vector<int2> cchild;
    std::vector<float> thr;
    for (auto &cs : v.codes) {
      if (cs.group >= 0) {
        const GroupItem &g = P.gitems[cs.group];
        cdesc.push_back(make_int4(sl(g.col), g.kind, (int)thr.size(), (int)g.thr.size()));
        thr.insert(thr.end(), g.thr.begin(), g.thr.end());
        cchild.push_back(make_int2(0, 0));
      } else {
        int ci = (int)(std::find(t.children[r].begin(), t.children[r].end(), cs.child_rel) - t.children[r].begin());
        cdesc.push_back(make_int4(-1, 0, 0, 0));
        cchild.push_back(make_int2(ci, cs.child_code));
      }
    }
    d.ncolsin = (int)slot.size();
    d.v64 = v.v64;
    d.codes = v.vcodes;
    d.ncols = (int)v.cols.size();
    d.ncodes = (int)v.codes.size();
    d.unique = v.unique_keys ? 1 : 0;
    d.nfac = (int)facs.size();
    v.keyrow = nullptr;
    if (v.unique_keys && v.nkeys < (int64_t(1) << 31) && Rr.nrows < (int64_t(1) << 31) &&
        view_key_rows_smem(d) <= 48 * 1024) {
      // the row of each key: the view is then computed key by key (coalesced, no memset)
      std::vector<DCol> kcols;
      for (int c : v.keycols) kcols.push_back(dcol(Rr.cols[c]));
      std::vector<int64_t> kst(d.kstride, d.kstride + d.nk);
      v.keyrow = (int *)P.arena.alloc(v.nkeys * 4 + 16);
      LMFAO_CUDA(cudaMemsetAsync(v.keyrow, 0xff, v.nkeys * 4 + 16, s));
      launch_key_rows(kcols.data(), (int)kcols.size(), P.arena.upload(kst, s), Rr.nrows, v.keyrow, s);
    }
    d.keyrow = v.keyrow;
    d.nkeys = v.nkeys;
    // unique keys and no children: the view kernel generated for these columns (LMFAO_CODEGEN=0
    // keeps the built-in one)
    GenView gv;
    const char *cg = std::getenv("LMFAO_CODEGEN");
    if (v.keyrow && !(cg && std::atoi(cg) == 0)) gv = gen_view(d, cfo, facs, cdesc, thr);
    P.vgen.push_back(gv);
    d.col_fac_off = P.arena.upload(cfo, s);
    d.facs = P.arena.upload(facs, s);
    d.col_part_off = P.arena.upload(cpo, s);
    d.parts = P.arena.upload(parts, s);
    d.code_desc = P.arena.upload(cdesc, s);
    d.code_child = P.arena.upload(cchild, s);
    d.thr = P.arena.upload(thr, s);
    d.err = P.err;
    P.vk.push_back(d);
    P.vk_rel.push_back(r);
    v.intcols_dev = icd;
    P.kernel_names.push_back("view:" + Rr.name);
  }
}

}  // namespace

// ======================================================================================
// root relation: reorganisation into segments, fact pass and combine descriptors
// ======================================================================================
namespace {

constexpr int64_t WORK_CHUNK = 4096;  // tuples per work item (segments longer than this split)

// Work items of the root pass: each segment in pieces of at most P.work_chunk tuples.
void build_work(lmfao_ctx *ctx, PhysPlan &P) {
  std::vector<DWork> work;
  long long r0 = 0;
  const int64_t wc = std::max(1, P.work_chunk);
  for (int64_t sidx = 0; sidx < P.nseg; ++sidx) {
    int64_t len = P.seg_hist[sidx];
    for (int64_t o = 0; o < len; o += wc)
      work.push_back(DWork{r0 + o, (int)sidx, (int)std::min<int64_t>(wc, len - o)});
    r0 += len;
  }
  P.nwork = (int64_t)work.size();
  P.work = P.arena.upload(work.empty() ? std::vector<DWork>{DWork{0, 0, 0}} : work, ctx->stream);
  if (work.empty()) P.nwork = 0;
  // tuple quantiles: q[j] = first item whose r0 >= ceil(j * total / kWorkQ)
  std::vector<int> q(kWorkQ + 1);
  const long long total = r0;
  size_t i = 0;
  for (int j = 0; j <= kWorkQ; ++j) {
    const long long at = (long long)(((__int128)total * j + kWorkQ - 1) / kWorkQ);
    while (i < work.size() && work[i].r0 < at) ++i;
    q[j] = (int)i;
  }
  q[kWorkQ] = (int)work.size();
  P.work_q = P.arena.upload(q, ctx->stream);
}

void setup_root(lmfao_ctx *ctx, PhysPlan &P, const JoinTree &t) {
  cudaStream_t s = ctx->stream;
  const Relation &F = ctx->rels[t.root];
  const int64_t n = F.nrows;
  const auto t0 = std::chrono::steady_clock::now();
  // reorganised copies of the root columns read per tuple, cached per (root, segment key)
  std::vector<int64_t> hist(P.nseg, 0);
  P.rowdev.clear();
  P.reorg_cached = false;
  if (P.segrel >= 0 && n > 0) {
    if (n >= (int64_t(1) << 32)) throw Error(LMFAO_ERR_UNSUPPORTED, "root relation of 2^32 tuples or more");
    lmfao_reorg *E = nullptr;
    for (auto &e : ctx->reorg)
      if (e.root == t.root && e.segcols == P.segcols) E = &e;
    std::vector<int> missing;
    for (int c : P.rowcols)
      if (!E || !E->cols.count(c)) missing.push_back(c);
    auto out_cols = [&](std::vector<DCol> &in, std::vector<DCol> &out, std::vector<int> &esz, lmfao_reorg &R) {
      for (int c : missing) {
        const Column &col = F.cols[c];
        const int e = col.dtype == LMFAO_U8 ? 1 : 4;
        void *p = nullptr;
        LMFAO_CUDA(cudaMalloc(&p, n * e + 16));  // padded: 4-tuple vector loads may read past the end
        LMFAO_CUDA(cudaMemsetAsync(p, 0, n * e + 16, s));
        R.cols[c] = p;
        in.push_back(dcol(col));
        out.push_back(DCol{p, col.dtype});
        esz.push_back(e);
      }
    };
    if (!E) {
      std::vector<DCol> kc;
      std::vector<int64_t> radix(P.segcols.size());
      int64_t acc = 1;
      for (int i = (int)P.segcols.size() - 1; i >= 0; --i) { radix[i] = acc; acc *= P.segdom[i]; }
      for (int c : P.segcols) kc.push_back(dcol(F.cols[c]));
      if (kc.size() > 4) throw Error(LMFAO_ERR_UNSUPPORTED, "segment key with more than 4 attributes");
      ctx->reorg.emplace_back();
      E = &ctx->reorg.back();
      E->root = t.root;
      E->segcols = P.segcols;
      LMFAO_CUDA(cudaMalloc((void **)&E->dest, n * 4));
      int *segid = (int *)P.arena.alloc(n * 4);
      unsigned int *h = (unsigned int *)P.arena.alloc(P.nseg * 4);
      LMFAO_CUDA(cudaMemsetAsync(h, 0, P.nseg * 4, s));
      launch_segment_ids(kc.data(), (int)kc.size(), radix.data(), n, segid, s);
      launch_histogram(segid, n, h, s);
      std::vector<unsigned int> hh(P.nseg);
      LMFAO_CUDA(cudaMemcpyAsync(hh.data(), h, P.nseg * 4, cudaMemcpyDeviceToHost, s));
      LMFAO_CUDA(cudaStreamSynchronize(s));
      std::vector<unsigned long long> begin(P.nseg);
      unsigned long long run = 0;
      E->hist.assign(P.nseg, 0);
      for (int64_t i = 0; i < P.nseg; ++i) { begin[i] = run; run += hh[i]; E->hist[i] = hh[i]; }
      unsigned long long *cursor = P.arena.upload(begin, s);
      std::vector<DCol> in, out;
      std::vector<int> esz;
      out_cols(in, out, esz, *E);
      // one pass assigns every row its position (kept for later columns) and moves the columns
      launch_scatter_rows(segid, n, cursor, in.data(), out.data(), esz.data(), (int)in.size(), E->dest, s);
      LMFAO_CUDA(cudaStreamSynchronize(s));
      cudaFree(segid);
      P.arena.ptrs.erase(std::find(P.arena.ptrs.begin(), P.arena.ptrs.end(), (void *)segid));
    } else {
      P.reorg_cached = missing.empty();
      std::vector<DCol> in, out;
      std::vector<int> esz;
      out_cols(in, out, esz, *E);
      launch_permute_rows(E->dest, n, in.data(), out.data(), esz.data(), (int)in.size(), s);
      LMFAO_CUDA(cudaStreamSynchronize(s));
    }
    hist = E->hist;
    for (int c : P.rowcols) P.rowdev.push_back(DCol{E->cols[c], F.cols[c].dtype});
  } else {
    hist[0] = n;
    for (int c : P.rowcols) P.rowdev.push_back(dcol(F.cols[c]));
  }
  P.reorg_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  P.seg_hist = hist;
  P.work_chunk = (int)WORK_CHUNK;
  build_work(ctx, P);
}

// Device tables of the specialised root pass and of the B3 finalisation.
void setup_fast(lmfao_ctx *ctx, PhysPlan &P, const JoinTree &t, DCombine &cb) {
  cudaStream_t s = ctx->stream;
  auto &F = P.fast;
  DFast &d = P.fd;
  d = DFast{};
  const size_t ts = P.fp64 ? 8 : 4;
  d.nwork = P.nwork;
  d.work = P.work;
  d.work_q = P.work_q;
  d.wseg = P.wseg;
  d.ncols = (int)P.rowdev.size();
  for (size_t i = 0; i < P.rowdev.size(); ++i) d.col[i] = P.rowdev[i];
  d.ni = (int)P.inner.size();
  std::vector<int> codecol;  // inner view code indices staged with the table
  auto code_pos = [&](int b) {
    for (size_t i = 0; i < codecol.size(); ++i) if (codecol[i] == b) return (int)i;
    codecol.push_back(b);
    return (int)codecol.size() - 1;
  };
  const View *iv = d.ni ? &P.views[P.inner[0]] : nullptr;
  if (iv) {
    DViewRef r = view_ref(*iv);
    d.nk = (int)iv->keycols.size();
    for (int i = 0; i < d.nk; ++i) { d.kslot[i] = P.rowslot.at(iv->pkeycols[i]); d.kstride[i] = r.kstride[i]; }
    d.nkeys = iv->nkeys;
  }
  d.nw = (int)F.wcols.size();
  // monomials as exponent tables over the loaded root columns, plus indicator factors
  std::vector<int> xslot;
  d.nm = (int)F.monos.size();
  std::memset(d.mexp, 0, sizeof(d.mexp));
  d.nind = 0;
  for (int j = 0; j < d.nm; ++j) {
    for (int f : F.monos[j]) {
      const Fac &fc = P.facs[f];
      int slot = P.rowslot.at(fc.col);
      if (fc.ind) {
        if (d.nind >= FMAXF) throw Error(LMFAO_ERR_UNSUPPORTED, "internal: too many indicator factors");
        d.ind[d.nind] = DFac{slot, 1, 1, fc.op, fc.t};
        d.ind_mono[d.nind] = j;
        ++d.nind;
        continue;
      }
      auto it = std::find(xslot.begin(), xslot.end(), slot);
      int xi;
      if (it == xslot.end()) {
        if ((int)xslot.size() >= FMAXX) throw Error(LMFAO_ERR_UNSUPPORTED, "internal: too many fact columns");
        xslot.push_back(slot);
        xi = (int)xslot.size() - 1;
      } else xi = (int)(it - xslot.begin());
      int e2 = d.mexp[j][xi] + fc.pow;
      if (e2 > 255) throw Error(LMFAO_ERR_UNSUPPORTED, "exponent too large");
      d.mexp[j][xi] = (unsigned char)e2;
    }
  }
  d.nx = (int)xslot.size();
  for (size_t i = 0; i < xslot.size(); ++i) d.xslot[i] = xslot[i];
  // B0
  d.n0i = (int)F.int0.size();
  for (int i = 0; i < d.n0i; ++i) { d.i0j[i] = F.int0[i].first; d.i0w[i] = F.int0[i].second; }
  P.phi0f = P.arena.alloc(std::max<size_t>(1, (size_t)P.nseg * d.nm * d.nw) * ts);
  P.phi0i = (unsigned long long *)P.arena.alloc(std::max<size_t>(1, (size_t)P.nseg * d.n0i) * 8);
  d.phi0f = P.phi0f;
  d.phi0i = P.phi0i;
  // B1
  d.nb1 = (int)F.b1.size();
  int64_t segf = 0, segi = 0;
  P.b1sets.clear();
  for (int si = 0; si < d.nb1; ++si) {
    auto &S = F.b1[si];
    DFastB1 &b = d.b1[si];
    b = DFastB1{};
    b.G = (int)S.G;
    b.nref = (int)S.refs.size();
    int64_t radix = 1;
    DB1Set cs{};
    cs.G = b.G;
    cs.nref = b.nref;
    for (int i = b.nref - 1; i >= 0; --i) {
      b.ref[i] = S.refs[i];
      b.ref[i].stride = radix;
      if (S.refs[i].src == 3) b.ref[i].b = code_pos(S.refs[i].b);
      cs.radix[i] = radix;
      cs.dom[i] = S.dom[i];
      radix *= S.dom[i];
    }
    b.nf = (int)S.fcols.size();
    b.ni = (int)S.icols.size();
    for (int c = 0; c < b.nf; ++c) { b.fj[c] = S.fcols[c].first; b.fw[c] = S.fcols[c].second; }
    for (int c = 0; c < b.ni; ++c) { b.ij[c] = S.icols[c].first; b.iw[c] = S.icols[c].second; }
    b.smem_f = d.hist_f;
    b.smem_i = d.hist_i;
    d.hist_f += b.G * b.nf;
    d.hist_i += b.G * b.ni;
    b.gbase_f = segf;
    b.gbase_i = segi;
    cs.nf = b.nf;
    cs.ni = b.ni;
    cs.gbase_f = segf;
    cs.gbase_i = segi;
    segf += (int64_t)b.G * b.nf;
    segi += (int64_t)b.G * b.ni;
    P.b1sets.push_back(cs);
  }
  d.phi1f_seg = segf;
  d.phi1i_seg = segi;
  d.lean = F.lean ? 1 : 0;
  d.vec = (P.segrel >= 0 && d.nk <= 1) ? 1 : 0;  // reorganised (padded) root columns
  for (int si = 0; si < d.nb1; ++si) d.b1code[si] = d.b1[si].ref[0].b;
  if ((double)P.nseg * (segf + segi) * 4 > 6e9) throw Error(LMFAO_ERR_UNSUPPORTED, "grouped per-segment sums exceed 6 GB");
  d.phi1f = (float *)P.arena.alloc(std::max<size_t>(1, (size_t)P.nseg * segf) * 4);
  d.phi1i = (unsigned int *)P.arena.alloc(std::max<size_t>(1, (size_t)P.nseg * segi) * 4);
  // B3
  d.n3 = (int)F.p3.size();
  d.n3f = d.n3i = 0;
  for (int c = 0; c < d.n3; ++c) {
    d.j3[c] = F.p3[c].first;
    d.int3[c] = F.p3[c].second ? 1 : 0;
    d.p3col[c] = d.int3[c] ? d.n3i++ : d.n3f++;
  }
  for (auto &b3 : F.b3) b3.c = d.p3col[b3.c];
  int64_t nk3 = std::max<int64_t>(1, d.nkeys);
  const int lsplit = std::max(1, F.b3leaf);
  d.p3f = (double *)P.arena.alloc((size_t)nk3 * std::max(1, d.n3f) * lsplit * 8);
  d.p3f32 = (float *)P.arena.alloc((size_t)nk3 * std::max(1, d.n3f) * lsplit * 4);
  d.p3i = (unsigned long long *)P.arena.alloc((size_t)nk3 * std::max(1, d.n3i) * lsplit * 8);
  d.ticket = (unsigned int *)P.arena.alloc(16);
  d.thr = cb.thr;
  // inner view table (staged per run by fast_prep) and codes
  for (auto &b3 : F.b3) (void)b3;
  // filter family: predicate bits per segment (outer), per inner key (inner), per tuple (root)
  d.nfam = F.fam_k;
  d.b3leaf = std::max(1, F.b3leaf);
  d.ibit_code = -1;
  d.nob = d.nrb = 0;
  std::vector<int2> ibits;
  if (d.nfam) {
    for (int f = 0; f < d.nfam; ++f) d.fmask[f] = F.fmask[f];
    for (auto &b : F.obits) {
      d.obit_outer[d.nob] = b[0];
      d.obit_col[d.nob] = b[1];
      d.obit_pos[d.nob] = b[2];
      ++d.nob;
    }
    for (auto &b : F.rbits) {
      const Fac &fc = P.facs[b[2]];
      d.rb[d.nrb] = DFac{b[0], 1, 1, fc.op, fc.t};
      d.rb_pos[d.nrb] = b[1];
      ++d.nrb;
    }
    for (auto &b : F.ibits) ibits.push_back(make_int2(b[0], b[1]));
    if (!ibits.empty()) {
      d.ibit_code = (int)codecol.size();
      codecol.push_back(-1);
    }
    d.nouter = cb.nouter;
    for (int o = 0; o < cb.nouter; ++o) d.outer[o] = cb.outer[o];
    d.seg = cb.seg;
  }
  P.fibits_dev = P.arena.upload(ibits.empty() ? std::vector<int2>{make_int2(0, 0)} : ibits, s);
  P.fnibits = (int)ibits.size();
  if (d.b3leaf > 1) {
    for (auto &b3 : F.b3) b3.c = b3.c * d.b3leaf + b3.leaf;  // already within-kind index
  }
  // B4: CTA-private outputs mirrored in shared memory per query region
  d.nb4 = (int)F.b4.size();
  {
    // order the items by filter index: items of every filter (sel -1) first
    std::stable_sort(F.b4.begin(), F.b4.end(), [](const PhysPlan::Fast::B4 &a, const PhysPlan::Fast::B4 &b) {
      return a.sel < b.sel;
    });
    for (int f = 0; f < FMAXFAM + 2; ++f) d.b4_off[f] = 0;
    for (int f = -1; f <= FMAXFAM; ++f) {
      int cnt = 0;
      for (auto &b : F.b4) cnt += b.sel < f ? 1 : 0;
      if (f + 1 < FMAXFAM + 2) d.b4_off[f + 1] = cnt;
    }
    std::vector<DGroupRef> g4;
    std::vector<DMirror> mir;
    std::map<std::pair<int, int>, int> base;  // (query, integral) -> shared offset
    int fcells = 0, icells = 0;
    for (int i = 0; i < d.nb4; ++i) {
      const auto &b = F.b4[i];
      const QueryOut &q = P.qout[b.q];
      const int64_t gbase = b.integral ? q.io : q.fo;
      const int64_t len = b.integral ? q.cells * (1 + q.naggs) : q.cells * q.naggs;
      auto key = std::make_pair(b.q, b.integral);
      auto it = base.find(key);
      if (it == base.end()) {
        int &cells = b.integral ? icells : fcells;
        mir.push_back(DMirror{gbase, cells, (int)len, b.integral, 0});
        it = base.emplace(key, cells).first;
        cells += (int)len;
      }
      d.b4_j[i] = b.j;
      d.b4_w[i] = b.w;
      d.b4_int[i] = b.integral;
      d.b4_sel[i] = b.sel;
      d.b4_g0[i] = (int)g4.size();
      d.b4_ng[i] = (int)b.refs.size();
      for (DGroupRef g : b.refs) {
        if (g.src == 3) g.b = code_pos(g.b);  // inner view code staged with the inner table
        g4.push_back(g);
      }
      d.b4_so[i] = it->second + (int)(b.out - gbase);
      d.b4_cellmul[i] = b.cellmul;
    }
    if (fcells + icells > 24 * 1024) throw Error(LMFAO_ERR_UNSUPPORTED, "internal: per-CTA outputs too large");
    d.b4_fcells = fcells;
    d.b4_icells = icells;
    d.nb4mirror = (int)mir.size();
    d.b4mirror = P.arena.upload(mir.empty() ? std::vector<DMirror>{DMirror{}} : mir, s);
    d.grefs4 = P.arena.upload(g4.empty() ? std::vector<DGroupRef>{DGroupRef{}} : g4, s);
    d.fsum = P.fsum;
    d.icnt = P.icnt;
  }
  d.ncode = (int)codecol.size();
  void *table = P.arena.alloc((size_t)nk3 * std::max(1, d.nw) * ts);
  int *codes = (int *)P.arena.alloc((size_t)nk3 * std::max(1, d.ncode) * 4);
  d.table = table;
  d.codes = codes;
  P.fwcol_dev = P.arena.upload(F.wcols, s);
  P.fcodecol_dev = P.arena.upload(codecol.empty() ? std::vector<int>{0} : codecol, s);
  // shared memory: the table and the B3 partials when they fit (1 CTA of 512 threads per SM)
  P.fast_block = P.fp64 ? 256 : 512;
  size_t pbytes = (ts * (size_t)d.nkeys * d.n3f + 4 * (size_t)d.nkeys * d.n3i) * lsplit;
  size_t vbytes = d.ni ? ts * (size_t)d.nkeys * d.nw + 4 * (size_t)d.nkeys * d.ncode : 0;
  size_t hbytes = (size_t)(P.fast_block / 32) * (d.hist_f + d.hist_i) * 4 + (ts * d.b4_fcells + 4 * d.b4_icells) + 64;
  if (hbytes > 96 * 1024) throw Error(LMFAO_ERR_UNSUPPORTED, "internal: group histograms too large");
  d.smem_p = d.n3 && pbytes + hbytes <= 190 * 1024 ? 1 : 0;
  d.smem_view = d.ni && vbytes + (d.smem_p ? pbytes : 0) + hbytes <= 190 * 1024 ? 1 : 0;
  size_t sm = fast_smem(d, P.fp64, P.fast_block);
  P.fast_grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm > 100 * 1024 ? 148 : 296, (P.nwork + 15) / 16));
  // plan-specialised kernel (code generation) for large root relations; LMFAO_CODEGEN=0
  // disables it, =1 forces it at any size
  P.gen = GenRootPass{};
  {
    const char *lanes = std::getenv("LMFAO_ROOT_LANES");
    d.lanes = lanes ? (std::atoi(lanes) != 0) : 0;
    const char *env = std::getenv("LMFAO_CODEGEN");
    const int mode = env ? std::atoi(env) : -1;
    if (mode == 1 || (mode != 0 && ctx->rels[P.root].nrows >= (int64_t(1) << 20))) {
      P.gen = gen_root_pass(d, P.fp64, ctx->device, P.thr);
      if (P.gen.fn) {
        int per_sm = 1, nsm = 148;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.gen.fn, P.gen.block, P.gen.smem);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
        cudaGetLastError();
        P.fast_grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(1, per_sm), P.nwork));
      }
    } else {
      P.gen.why = mode == 0 ? "disabled" : "root relation below 2^20 tuples";
    }
  }
  // B3 finalisation
  DB3Final &f = P.b3f;
  f = DB3Final{};
  if (iv) {
    f.nkeys = iv->nkeys;
    f.v64 = iv->v64;
    f.vcols = (int)iv->cols.size();
    f.vcodes = iv->vcodes;
    f.vncodes = (int)iv->codes.size();
  }
  f.p3f = d.p3f;
  f.p3i = d.p3i;
  f.p3f32 = (d.smem_p || P.fp64) ? nullptr : d.p3f32;  // FP64 plans keep FP64 global partials
  f.n3 = d.n3;
  f.n3f = d.n3f * lsplit;
  f.n3i = d.n3i * lsplit;
  f.nitems = (int)F.b3.size();
  f.items = P.arena.upload(F.b3, s);
  f.grefs = cb.grefs;
  f.fsum = P.fsum;
  f.icnt = P.icnt;
  // combine reads the specialised PHI layout
  cb.n0f = d.nm * d.nw;
  cb.n0i = d.n0i;
  cb.phi0f = P.phi0f;
  cb.phi0i = P.phi0i;
  cb.nsets = (int)P.b1sets.size();
  cb.sets = P.arena.upload(P.b1sets, s);
  cb.phi1f = d.phi1f;
  cb.phi1i = d.phi1i;
  cb.phi1f_seg = segf;
  cb.phi1i_seg = segi;
  (void)t;
}

// Entries, staged columns and outer-cell sets of the combine (combine.cu).
void setup_combine2(lmfao_ctx *ctx, PhysPlan &P, const std::vector<DPart> &pparts) {
  cudaStream_t s = ctx->stream;
  const DCombine &cb = P.cb;
  DComb2 &d = P.c2;
  d = DComb2{};
  d.nseg = P.nseg;
  d.wseg = P.wseg;
  d.seg = cb.seg;
  d.nouter = cb.nouter;
  for (int i = 0; i < cb.nouter; ++i) d.outer[i] = cb.outer[i];
  // staged outer view columns
  std::vector<int2> stage;
  std::vector<int> psi_stage;
  for (const DPart &pp : pparts) {
    int at = -1;
    for (size_t i = 0; i < stage.size(); ++i)
      if (stage[i].x == pp.branch && stage[i].y == pp.col) at = (int)i;
    if (at < 0) { stage.push_back(make_int2(pp.branch, pp.col)); at = (int)stage.size() - 1; }
    psi_stage.push_back(at);
  }
  d.nstage = (int)stage.size();
  d.stage_col = P.arena.upload(stage.empty() ? std::vector<int2>{make_int2(0, 0)} : stage, s);
  d.npsi = cb.npsi;
  d.psi = cb.psi;
  d.segfacs = cb.segfacs;
  d.psi_stage = P.arena.upload(psi_stage.empty() ? std::vector<int>{0} : psi_stage, s);
  // outer-cell sets
  std::vector<std::vector<DGroupRef>> ogs{{}};
  auto same = [](const DGroupRef &a, const DGroupRef &b) {
    return a.src == b.src && a.a == b.a && a.b == b.b && a.stride == b.stride;
  };
  auto og_of = [&](const DCombItem &it) {
    std::vector<DGroupRef> g(P.grefs.begin() + it.og0, P.grefs.begin() + it.og0 + it.nog);
    for (size_t i = 0; i < ogs.size(); ++i) {
      if (ogs[i].size() != g.size()) continue;
      bool eq = true;
      for (size_t j = 0; j < g.size(); ++j) eq = eq && same(ogs[i][j], g[j]);
      if (eq) return (int)i;
    }
    ogs.push_back(g);
    return (int)ogs.size() - 1;
  };
  // Y columns
  d.n0f = cb.n0f;
  d.n0i = cb.n0i;
  int64_t segf = P.fast.on ? P.fd.phi1f_seg : 0, segi = P.fast.on ? P.fd.phi1i_seg : 0;
  d.nyf = (int)(d.n0f + segf);
  d.nyi = (int)(d.n0i + segi);
  d.phi0f = cb.phi0f;
  d.phi0i = cb.phi0i;
  d.phi1f = P.fast.on ? P.fd.phi1f : nullptr;
  d.phi1i = P.fast.on ? P.fd.phi1i : nullptr;
  d.phi1f_seg = segf;
  d.phi1i_seg = segi;
  // mirrors: query output regions of entries whose cell varies, while they fit
  std::vector<DMirror> mirrors;
  std::map<int64_t, int> fmir, imir;
  int fcells = 0, icells = 0;
  const int budget = 10 * 1024;
  auto mirror_of = [&](const DCombItem &it) -> int {
    if (it.nog == 0 && it.block < 0) return -1;
    for (auto &q : P.qout) {
      int64_t base = it.integral ? q.io : q.fo;
      int64_t len = it.integral ? q.cells * (1 + q.naggs) : q.cells * q.naggs;
      if (it.out < base || it.out >= base + len) continue;
      auto &mp = it.integral ? imir : fmir;
      int &cells = it.integral ? icells : fcells;
      auto f = mp.find(base);
      if (f == mp.end()) {
        if (cells + len > budget) return -1;
        mp[base] = cells;
        mirrors.push_back(DMirror{base, cells, (int)len, it.integral, 0});
        f = mp.find(base);
        cells += (int)len;
      }
      return f->second + (int)(it.out - base);
    }
    return -1;
  };
  std::vector<DEntry> ent;
  for (const DCombItem &it : P.comb) {
    int og = og_of(it);
    int so = mirror_of(it);
    if (it.block < 0) {
      DEntry e{};
      e.psi = it.psi;
      e.ycol = it.col;
      e.og = og;
      e.integral = it.integral;
      e.so = so;
      e.out = it.out;
      e.cellmul = it.cellmul;
      e.icell = 0;
      ent.push_back(e);
    } else {
      const DB1Set &S = P.b1sets[it.block];
      const auto &srefs = P.fast.b1[it.block].refs;
      for (int g = 0; g < S.G; ++g) {
        bool pick = true;
        for (int i = 0; i < S.nref; ++i)
          if (srefs[i].src == 4 && (g / S.radix[i]) % S.dom[i] != it.sel) pick = false;
        if (!pick) continue;
        DEntry e{};
        e.psi = it.psi;
        e.ycol = it.yint ? (int)(d.n0i + S.gbase_i + (int64_t)g * S.ni + it.col)
                         : (int)(d.n0f + S.gbase_f + (int64_t)g * S.nf + it.col);
        e.yint = it.yint;
        e.og = og;
        e.integral = it.integral;
        e.so = so;
        e.out = it.out;
        e.cellmul = it.cellmul;
        int64_t ic = 0;
        for (int i = 0; i < S.nref; ++i) ic += ((g / S.radix[i]) % S.dom[i]) * P.grefs[it.ig0 + i].stride;
        e.icell = ic;
        ent.push_back(e);
      }
    }
  }
  std::vector<int> og_off{0};
  std::vector<DGroupRef> og_refs;
  for (auto &g : ogs) {
    og_refs.insert(og_refs.end(), g.begin(), g.end());
    og_off.push_back((int)og_refs.size());
  }
  d.nog = (int)ogs.size();
  d.og_off = P.arena.upload(og_off, s);
  d.grefs = P.arena.upload(og_refs.empty() ? std::vector<DGroupRef>{DGroupRef{}} : og_refs, s);
  d.nent = (int)ent.size();
  d.ent = P.arena.upload(ent.empty() ? std::vector<DEntry>{DEntry{}} : ent, s);
  d.nmirror = (int)mirrors.size();
  d.mirror = P.arena.upload(mirrors.empty() ? std::vector<DMirror>{DMirror{}} : mirrors, s);
  d.mirror_f = fcells;
  d.mirror_i = icells;
  d.fsum = P.fsum;
  d.icnt = P.icnt;
  d.tile = 16;
  while (d.tile > 1 && combine2_smem(d, P.fp64) > 200 * 1024) d.tile /= 2;
  if (combine2_smem(d, P.fp64) > 220 * 1024) throw Error(LMFAO_ERR_UNSUPPORTED, "combine needs too much shared memory");
  P.c2_block = 512;
  size_t sm = combine2_smem(d, P.fp64);
  int per_sm = sm > 110 * 1024 ? 1 : 2;
  int64_t ranges = std::max<int64_t>(1, std::min<int64_t>(148 * per_sm, (P.nseg + d.tile - 1) / d.tile));
  P.c2_grid = (int)ranges;
  P.c2h_ent = ent;
  P.c2h_og_off = og_off;
  P.c2h_og_refs = og_refs;
}

// Projection combine (combine4.cu): eligible for a two-digit segment key when every outer
// cell is a segment digit or an outer view code and the cells of an entry fit a CTA.
// Returns false otherwise (the entry combine runs).
bool setup_combine4(lmfao_ctx *ctx, PhysPlan &P, const std::vector<DPsi> &psi, const std::vector<DSegFac> &segfacs,
                    const std::vector<DPart> &pparts) {
  cudaStream_t s = ctx->stream;
  const DComb2 &c2 = P.c2;
  const std::vector<DEntry> &ent = P.c2h_ent;
  const std::vector<int> &og_off = P.c2h_og_off;
  const std::vector<DGroupRef> &og_refs = P.c2h_og_refs;
  if (std::getenv("LMFAO_NO_PROJECTION_COMBINE")) return false;
  if (c2.seg.ndig != 2 || ent.empty() || c2.seg.radix[1] != 1 || c2.seg.radix[0] != c2.seg.dom[1]) return false;
  auto outer_digits = [&](int o) {
    unsigned m = 0;
    for (int i = 0; i < 2; ++i)
      if (c2.outer[o].dstride[i]) m |= 1u << i;
    return m;
  };
  // when every outer view holds at most one tuple per key, its COUNT is 1 on every live
  // segment and the COUNT parts of an outer term depend on no digit
  bool skip_counts = true;
  for (int c : P.outer) skip_counts = skip_counts && P.views[c].count_bound <= 1.0;
  auto psi_digits = [&](int t) {
    unsigned m = 0;
    const DPsi &p = psi[t];
    for (int f = p.f0; f < p.f0 + p.nf; ++f) m |= 1u << segfacs[f].digit;
    for (int i = p.p0; i < p.p0 + p.np; ++i)
      if (!(skip_counts && pparts[i].col == 0)) m |= outer_digits(pparts[i].branch);
    return m;
  };
  const int nog = (int)og_off.size() - 1;
  std::vector<unsigned> og_dig(nog, 0);
  for (int g = 0; g < nog; ++g)
    for (int r = og_off[g]; r < og_off[g + 1]; ++r) {
      const DGroupRef &q = og_refs[r];
      if (q.src == 0) og_dig[g] |= 1u << q.a;
      else if (q.src == 1) og_dig[g] |= outer_digits(q.a);
      else return false;
    }
  // compact cells of each outer-cell set (domains from the query of an entry that uses it)
  std::vector<long long> cstride(std::max<size_t>(1, og_refs.size()), 1), cdom(std::max<size_t>(1, og_refs.size()), 1);
  std::vector<long long> ncells(nog, 1);
  std::vector<bool> og_done(nog, false);
  for (const DEntry &e : ent) {
    if (og_done[e.og]) continue;
    int qi = -1;
    for (size_t k = 0; k < P.qout.size(); ++k) {
      const QueryOut &q = P.qout[k];
      const int64_t base = e.integral ? q.io : q.fo;
      const int64_t len = e.integral ? q.cells * (1 + q.naggs) : q.cells * q.naggs;
      if (e.out >= base && e.out < base + len) qi = (int)k;
    }
    if (qi < 0) return false;
    const QueryOut &q = P.qout[qi];
    std::vector<int64_t> qs(q.dom.size(), 1);
    for (int i = (int)q.dom.size() - 2; i >= 0; --i) qs[i] = qs[i + 1] * q.dom[i + 1];
    long long cs = 1;
    for (int r = og_off[e.og + 1] - 1; r >= og_off[e.og]; --r) {
      long long dm = 1;
      for (size_t i = 0; i < q.dom.size(); ++i)
        if (qs[i] == og_refs[r].stride && q.dom[i] > 1) dm = q.dom[i];
      cdom[r] = dm;
      cstride[r] = cs;
      cs *= dm;
    }
    ncells[e.og] = cs;
    og_done[e.og] = true;
  }
  // jobs (Y columns) and entry classes
  std::map<std::pair<int, int>, int> jobs;
  std::vector<int2> job;
  std::vector<DEntry4> e012[3], e3;
  long long max_cells = 1;
  for (const DEntry &e : ent) {
    const bool yint = e.integral || e.yint;
    auto key = std::make_pair(yint ? 1 : 0, e.ycol);
    auto it = jobs.find(key);
    if (it == jobs.end()) {
      it = jobs.emplace(key, (int)job.size()).first;
      job.push_back(make_int2(key.first, key.second));
    }
    const unsigned dep = psi_digits(e.psi) | og_dig[e.og];
    DEntry4 x{};
    x.psi = e.psi;
    x.og = e.og;
    x.cls = dep == 0 ? 0 : dep == 1 ? 1 : dep == 2 ? 2 : 3;
    x.flags = (e.integral ? 1 : 0) | (yint ? 2 : 0);
    x.job = it->second;
    x.out = e.out;
    x.cellmul = e.cellmul;
    x.icell = e.icell;
    if (x.cls == 3) {
      e3.push_back(x);
    } else {
      e012[x.cls].push_back(x);
      max_cells = std::max(max_cells, ncells[e.og]);
    }
  }
  if (max_cells > 6144) return false;
  const int nj = (int)job.size();
  std::stable_sort(e3.begin(), e3.end(), [](const DEntry4 &a, const DEntry4 &b) { return a.job < b.job; });
  // per-class tables of the outer terms and cells the entries read
  std::map<int, int> tm[4], gm[4];
  std::vector<int> tv[4], gv[4];
  auto tabulate = [&](DEntry4 &x) {
    const int c = x.cls == 0 ? 0 : x.cls;
    if (c == 0) return;
    auto ti = tm[c].find(x.psi);
    if (ti == tm[c].end()) { ti = tm[c].emplace(x.psi, (int)tv[c].size()).first; tv[c].push_back(x.psi); }
    auto gi = gm[c].find(x.og);
    if (gi == gm[c].end()) { gi = gm[c].emplace(x.og, (int)gv[c].size()).first; gv[c].push_back(x.og); }
    x.psi = ti->second;
    x.tog = gi->second;
  };
  for (DEntry4 &x : e3) tabulate(x);
  for (int c = 1; c < 3; ++c)
    for (DEntry4 &x : e012[c]) tabulate(x);
  // class 3 slots: per tile of 256 entries (one thread each), the cells of its entries
  int max_slots3 = 0;
  for (size_t i = 0, used = 0; i < e3.size(); ++i) {
    if (i % 256 == 0) used = 0;
    e3[i].sbase = (int)used;
    used += (size_t)ncells[e3[i].og];
    max_slots3 = std::max(max_slots3, (int)used);
  }
  if (max_slots3 > 12 * 1024) return false;
  // streaming form: every class 3 entry's cells after those of the entries before it
  long long nslots3 = 0;
  for (DEntry4 &x : e3) {
    x.pad = (int)nslots3;
    nslots3 += ncells[x.og];
  }
  std::vector<int> e3_off(nj + 1, 0);
  for (const DEntry4 &x : e3) e3_off[x.job + 1]++;
  for (int j = 0; j < nj; ++j) e3_off[j + 1] += e3_off[j];
  std::vector<DEntry4> all;
  for (int c = 0; c < 3; ++c) all.insert(all.end(), e012[c].begin(), e012[c].end());
  DComb4 &d = P.c4;
  d = DComb4{};
  d.c = c2;
  d.dom0 = (int)c2.seg.dom[0];
  d.dom1 = (int)c2.seg.dom[1];
  d.njobs = nj;
  d.job = P.arena.upload(job, s);
  d.nent012 = (int)all.size();
  d.ent = P.arena.upload(all.empty() ? std::vector<DEntry4>{DEntry4{}} : all, s);
  d.nent3 = (int)e3.size();
  d.ent3 = P.arena.upload(e3.empty() ? std::vector<DEntry4>{DEntry4{}} : e3, s);
  d.e3_off = P.arena.upload(e3_off, s);
  for (int c = 1; c <= 3; ++c) {
    DTab4 &tb = d.tab[c];
    const int64_t nv = c == 1 ? d.dom0 : c == 2 ? d.dom1 : P.nseg;
    tb.nt = (int)tv[c].size();
    tb.ng = (int)gv[c].size();
    tb.t = P.arena.upload(tv[c].empty() ? std::vector<int>{0} : tv[c], s);
    tb.g = P.arena.upload(gv[c].empty() ? std::vector<int>{0} : gv[c], s);
    tb.pf = (double *)P.arena.alloc((size_t)nv * std::max(1, tb.nt) * 8);
    tb.pi = (unsigned long long *)P.arena.alloc((size_t)nv * std::max(1, tb.nt) * 8);
    tb.cell = (long long *)P.arena.alloc((size_t)nv * std::max(1, tb.ng) * 8);
  }
  d.skip_counts = skip_counts ? 1 : 0;
  d.max_slots3 = max_slots3;
  d.need_d0 = e012[1].empty() ? 0 : 1;
  d.need_d1 = e012[2].empty() ? 0 : 1;
  d.yd0_f = (double *)P.arena.alloc((size_t)d.dom0 * nj * 8);
  d.yd0_i = (unsigned long long *)P.arena.alloc((size_t)d.dom0 * nj * 8);
  d.yd1_f = (double *)P.arena.alloc((size_t)d.dom1 * nj * 8);
  d.yd1_i = (unsigned long long *)P.arena.alloc((size_t)d.dom1 * nj * 8);
  d.yall_f = (double *)P.arena.alloc((size_t)nj * 8);
  d.yall_i = (unsigned long long *)P.arena.alloc((size_t)nj * 8);
  d.og_ncells = P.arena.upload(ncells, s);
  d.og_cstride = P.arena.upload(cstride, s);
  d.og_dom = P.arena.upload(cdom, s);
  d.max_cells = (int)max_cells;
  // streaming form for batches with few Y columns (a decision-tree level: 24), the separate
  // projection kernels for many (Favorita's 379, where the streaming form measured slower);
  // LMFAO_PROJECTION=stream|kernels overrides. Tiles of about 6,144 staged sums, about two CTAs
  // per SM, class 3 fused when its cells fit.
  d.nslots3 = (int)std::min<long long>(nslots3, 1 << 30);
  const char *pk = std::getenv("LMFAO_PROJECTION");
  d.stream = pk ? (std::string(pk) == "stream" ? 1 : 0) : (nj <= 64 ? 1 : 0);
  if (d.stream) {
    d.c1 = (int)std::max<int64_t>(1, std::min<int64_t>(d.dom1, (6144 + nj - 1) / std::max(1, nj)));
    while (d.c1 > 1 && 16 * (size_t)d.c1 * nj > 160 * 1024) d.c1 /= 2;
    d.nx = (d.dom1 + d.c1 - 1) / d.c1;
    int ny = (int)std::max<int64_t>(1, std::min<int64_t>(d.dom0, 296 / std::max(1, d.nx)));
    d.c0 = (d.dom0 + ny - 1) / ny;
    d.ny = (d.dom0 + d.c0 - 1) / d.c0;
    const size_t tab3 = (size_t)d.c1 * (2 * d.tab[3].nt + d.tab[3].ng);  // staged terms and cells of a row
    d.fused3 = d.nent3 > 0 && d.nent3 <= 512 && 8 * (2 * (size_t)d.c1 * nj + (size_t)nslots3 + tab3 + nj) <= 200 * 1024
                   ? 1 : 0;
    d.sblock = d.fused3 && d.nent3 > 256 ? 512 : 256;
    d.yd0p = (unsigned long long *)P.arena.alloc((size_t)d.nx * d.dom0 * nj * 8);
    d.yd1p = (unsigned long long *)P.arena.alloc((size_t)d.ny * d.dom1 * nj * 8);
  }
  P.use_c4 = true;
  return true;
}

// Two-kernel block combine (combine5.cu) over the block tables of P.c3: per-block contraction
// Z_p = B_p^T Y_p into a global scratch array (FP32/FP64 on the CUDA cores, or split BF16 on
// the tensor cores when the plan asks for it and Y and the B terms fit one MMA tile), then
// one pass over the entries. Returns false (with the reason in P.c5_why) when it does not
// apply; the single-kernel block combine then runs.
bool setup_combine5(lmfao_ctx *ctx, PhysPlan &P) {
  const char *env = getenv("LMFAO_COMBINE");
  if (env && std::string(env) == "single") {
    P.c5_why = "LMFAO_COMBINE=single";
    return false;
  }
  const DComb3 &d = P.c3;
  DComb5 D{};
  D.c = d;
  const int ny = d.nyf + d.nyi;
  const int64_t m = d.m;
  const bool tc_fits = ny <= 128 && d.nb <= 256;
  D.tc = P.split_bf16 && tc_fits ? 1 : 0;
  if (P.split_bf16 && !tc_fits)
    P.c5_why = "split BF16 needs at most 128 Y columns and 256 B terms (have " + std::to_string(ny) + ", " +
               std::to_string(d.nb) + "): contraction in FP32";
  D.npad = std::max(16, (d.nb + 15) / 16 * 16);
  D.tmem_cols = 32;
  while (D.tmem_cols < D.npad) D.tmem_cols *= 2;
  const int ts = P.fp64 ? 8 : 4;
  // CUDA cores with single-column B terms: the dense kernel (LMFAO_COMBINE=general keeps the
  // general one)
  D.dense = !D.tc && (int)P.c3_bsrc.size() == d.nb && d.nb > 0 && combine5_dense_fits(d) &&
            !(env && std::string(env) == "general");
  if (D.dense) D.bsrc = P.arena.upload(P.c3_bsrc, ctx->stream);
  // pipelined form: the B columns come from one outer view whose row for segment j of a block
  // is the block's row + j (its minor-digit strides equal the segment radices)
  if (D.dense && !(env && std::string(env) == "dense")) {
    int ob = -1;
    std::string why;
    for (const int2 &b : P.c3_bsrc)
      if (b.x >= 0) {
        if (ob < 0) ob = b.x;
        else if (ob != b.x) why = "B columns from several outer views";
      }
    if (ob < 0) why = "no B view column";
    // one minor digit (radix 1, domain m): segment j of a block reads the view row at the
    // block's row + j x the digit's stride in the view key
    int nminor = 0;
    int64_t bstride = 0;
    for (int i = 0; why.empty() && i < d.seg.ndig; ++i)
      if (d.seg.radix[i] < m) {
        ++nminor;
        bstride = d.outer[ob].dstride[i];
        if (d.seg.radix[i] != 1 || d.seg.dom[i] != m || bstride <= 0) why = "minor digit is not the whole block";
      }
    if (why.empty() && nminor != 1) why = "more than one minor digit";
    D.pipe = why.empty() ? 1 : 0;
    D.bout = why.empty() ? ob : 0;
    D.bstride = why.empty() ? bstride : 0;
    if (!why.empty()) P.c5_why = "pipelined contraction declined: " + why;
  }
  int kc0 = 64;
  if (const char *k = getenv("LMFAO_COMBINE_CHUNK")) kc0 = std::max(16, atoi(k) / 16 * 16);
  int kc = D.tc ? (int)std::min<int64_t>(kc0, (m + 15) / 16 * 16) : (int)std::min<int64_t>(kc0, m);
  for (; kc >= (D.tc ? 16 : 1); kc = D.tc ? kc - 16 : kc / 2) {
    D.kc = kc;
    if (combine5_smem(D, P.fp64) <= 200 * 1024) break;
  }
  if (kc < (D.tc ? 16 : 1)) {
    P.c5_why = "block tables do not fit shared memory";
    return false;
  }
  // TMA bulk staging: every chunk's rows start on a 16-byte boundary and span a multiple of 16 bytes
  const int64_t rb[5] = {(int64_t)d.n0f * ts, d.phi1f_seg * 4, (int64_t)d.n0i * 8, d.phi1i_seg * 4, 8};
  const void *base[5] = {d.phi0f, d.phi1f, d.phi0i, d.phi1i, d.wseg};
  D.bulk = D.dense ? 0 : 1;  // the dense kernel reads its operands with coalesced loads
  for (int i = 0; i < 5 && D.bulk; ++i) {
    if (!rb[i]) continue;
    if ((m * rb[i]) % 16 || ((int64_t)D.kc * rb[i]) % 16 || ((uintptr_t)base[i] % 16)) D.bulk = 0;
  }
  const int64_t nz = d.nblocks * (int64_t)d.nb * ny, nzi = d.nblocks * (int64_t)d.nbi * d.nyi;
  const int64_t bytes = nz * ts + nzi * 8 + d.nblocks * (int64_t)d.na * (ts + 8) + d.nblocks * (int64_t)d.nog * 8 +
                        d.nblocks * 4;
  if (bytes > ((int64_t)1 << 30)) {
    P.c5_why = "per-block scratch above 1 GiB";
    return false;
  }
  D.z = P.arena.alloc(std::max<int64_t>(1, nz) * ts);
  D.zi = (unsigned long long *)P.arena.alloc(std::max<int64_t>(1, nzi) * 8);
  D.a = P.arena.alloc(std::max<int64_t>(1, d.nblocks * (int64_t)d.na) * ts);
  D.ai = (unsigned long long *)P.arena.alloc(std::max<int64_t>(1, d.nblocks * (int64_t)d.na) * 8);
  D.cells = (long long *)P.arena.alloc(std::max<int64_t>(1, d.nblocks * (int64_t)d.nog) * 8);
  D.live = (int *)P.arena.alloc(std::max<int64_t>(1, d.nblocks) * 4);
  D.err = P.err;
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  D.grid = (int)std::min<int64_t>(d.nblocks, (int64_t)sms * 8);
  const int64_t ethreads = (int64_t)(d.nent + 255) / 256 * 256;
  D.eranges = (int)std::max<int64_t>(1, std::min<int64_t>(d.nblocks, ((int64_t)sms * 2048 + ethreads - 1) /
                                                                        std::max<int64_t>(1, ethreads)));
  (void)ctx;
  P.c5 = D;
  return true;
}

// Prefix-block combine (combine3.cu): eligible when the segment key has a proper prefix,
// every outer cell is constant inside a block (A-level group references only) and the
// block tables fit in shared memory. Returns false otherwise (the entry combine runs).
bool setup_combine3(lmfao_ctx *ctx, PhysPlan &P, const std::vector<DPsi> &psi, const std::vector<DSegFac> &segfacs,
                    const std::vector<DPart> &pparts) {
  cudaStream_t s = ctx->stream;
  const DCombine &cb = P.cb;
  const int L = P.prefix_len, nd = (int)P.segcols.size();
  if (L <= 0 || L >= nd || P.comb.empty()) return false;
  DComb3 d{};
  d.m = 1;
  for (int i = L; i < nd; ++i) d.m *= P.segdom[i];
  d.nblocks = P.nseg / d.m;
  if (d.m < 2) return false;
  d.wseg = P.wseg;
  d.seg = cb.seg;
  d.nouter = cb.nouter;
  std::vector<bool> aview(cb.nouter, true);
  for (int o = 0; o < cb.nouter; ++o) {
    d.outer[o] = cb.outer[o];
    for (int i = L; i < nd; ++i)
      if (cb.outer[o].dstride[i]) aview[o] = false;
  }
  // split every psi term into its prefix (A) part and its block-varying (B) part
  struct TermKey {
    std::vector<int> segf;
    std::vector<std::pair<int, int>> parts;
    bool operator<(const TermKey &o) const { return std::tie(segf, parts) < std::tie(o.segf, o.parts); }
  };
  auto integral_part = [&](int o, int col) { return P.views[P.outer[o]].cols[col].integral; };
  std::map<TermKey, int> amap, bmap;
  std::vector<TermKey> aterms, bterms;
  std::vector<bool> aint, bint;
  std::vector<int> psi_a(psi.size()), psi_b(psi.size());
  for (size_t t = 0; t < psi.size(); ++t) {
    TermKey ka, kb;
    bool ia = true, ib = true;
    for (int f = psi[t].f0; f < psi[t].f0 + psi[t].nf; ++f) {
      bool inA = segfacs[f].digit < L;
      (inA ? ka : kb).segf.push_back(f);
      if (!segfacs[f].ind) (inA ? ia : ib) = false;
    }
    for (int i = psi[t].p0; i < psi[t].p0 + psi[t].np; ++i) {
      const DPart &q = pparts[i];
      if (aview[q.branch]) { ka.parts.push_back({q.branch, q.col}); ia = ia && integral_part(q.branch, q.col); }
      else { kb.parts.push_back({q.branch, q.col}); ib = ib && integral_part(q.branch, q.col); }
    }
    auto put = [](std::map<TermKey, int> &mp, std::vector<TermKey> &v, std::vector<bool> &iv, const TermKey &k, bool in) {
      auto it = mp.find(k);
      if (it != mp.end()) return it->second;
      int id = (int)v.size();
      mp[k] = id;
      v.push_back(k);
      iv.push_back(in);
      return id;
    };
    psi_a[t] = put(amap, aterms, aint, ka, ia);
    psi_b[t] = put(bmap, bterms, bint, kb, ib);
  }
  // integral B terms first
  std::vector<int> border(bterms.size()), bpos(bterms.size());
  int nbi = 0;
  {
    int q = 0;
    for (size_t b = 0; b < bterms.size(); ++b) if (bint[b]) border[q++] = (int)b;
    nbi = q;
    for (size_t b = 0; b < bterms.size(); ++b) if (!bint[b]) border[q++] = (int)b;
    for (size_t i = 0; i < border.size(); ++i) bpos[border[i]] = (int)i;
  }
  auto stage_terms = [&](const std::vector<TermKey> &terms, const std::vector<int> &order, std::vector<int2> &stage,
                         std::vector<DPsi> &out, std::vector<int> &part, const std::vector<bool> &isint) {
    for (int ti : order) {
      const TermKey &k = terms[ti];
      DPsi dp{};
      dp.f0 = 0;
      dp.nf = 0;
      dp.p0 = (int)part.size();
      for (auto &pr : k.parts) {
        int at = -1;
        for (size_t i = 0; i < stage.size(); ++i) if (stage[i].x == pr.first && stage[i].y == pr.second) at = (int)i;
        if (at < 0) { stage.push_back(make_int2(pr.first, pr.second)); at = (int)stage.size() - 1; }
        part.push_back(at);
      }
      dp.np = (int)k.parts.size();
      dp.integral = isint[ti] ? 1 : 0;
      out.push_back(dp);
    }
  };
  // segment factors stay in the shared segfacs table: a term lists them as a contiguous run
  std::vector<DSegFac> sf2;
  auto with_segf = [&](std::vector<DPsi> &terms, const std::vector<TermKey> &keys, const std::vector<int> &order) {
    for (size_t i = 0; i < order.size(); ++i) {
      terms[i].f0 = (int)sf2.size();
      for (int f : keys[order[i]].segf) sf2.push_back(segfacs[f]);
      terms[i].nf = (int)keys[order[i]].segf.size();
    }
  };
  std::vector<int2> astage, bstage;
  std::vector<DPsi> adesc, bdesc;
  std::vector<int> apart, bpart;
  std::vector<int> aorder(aterms.size());
  std::iota(aorder.begin(), aorder.end(), 0);
  stage_terms(aterms, aorder, astage, adesc, apart, aint);
  stage_terms(bterms, border, bstage, bdesc, bpart, bint);
  with_segf(adesc, aterms, aorder);
  with_segf(bdesc, bterms, border);
  // B terms that are single view columns (or 1): the dense two-kernel contraction reads them
  P.c3_bsrc.clear();
  for (const DPsi &b : bdesc) {
    if (b.nf || b.np > 1) {
      P.c3_bsrc.clear();
      break;
    }
    P.c3_bsrc.push_back(b.np ? bstage[bpart[b.p0]] : make_int2(-1, -1));
  }
  // Y columns
  d.n0f = cb.n0f;
  d.n0i = cb.n0i;
  int64_t segf = P.fast.on ? P.fd.phi1f_seg : 0, segi = P.fast.on ? P.fd.phi1i_seg : 0;
  d.nyf = (int)(d.n0f + segf);
  d.nyi = (int)(d.n0i + segi);
  d.phi0f = cb.phi0f;
  d.phi0i = cb.phi0i;
  d.phi1f = P.fast.on ? P.fd.phi1f : nullptr;
  d.phi1i = P.fast.on ? P.fd.phi1i : nullptr;
  d.phi1f_seg = segf;
  d.phi1i_seg = segi;
  // outer-cell sets (A-level only) and entries
  std::vector<std::vector<DGroupRef>> ogs{{}};
  auto og_of = [&](const DCombItem &it) -> int {
    std::vector<DGroupRef> g(P.grefs.begin() + it.og0, P.grefs.begin() + it.og0 + it.nog);
    for (auto &r : g) {
      if (r.src == 0 && r.a >= L) return -1;
      if (r.src == 1 && !aview[r.a]) return -1;
    }
    for (size_t i = 0; i < ogs.size(); ++i) {
      if (ogs[i].size() != g.size()) continue;
      bool eq = true;
      for (size_t j = 0; j < g.size(); ++j)
        eq = eq && ogs[i][j].src == g[j].src && ogs[i][j].a == g[j].a && ogs[i][j].b == g[j].b &&
             ogs[i][j].stride == g[j].stride;
      if (eq) return (int)i;
    }
    ogs.push_back(g);
    return (int)ogs.size() - 1;
  };
  std::vector<DMirror> mirrors;
  std::map<int64_t, int> fmir, imir;
  int fcells = 0, icells = 0;
  auto mirror_of = [&](const DCombItem &it) -> int {
    if (it.nog == 0 && it.block < 0) return -1;
    for (auto &q : P.qout) {
      int64_t base = it.integral ? q.io : q.fo;
      int64_t len = it.integral ? q.cells * (1 + q.naggs) : q.cells * q.naggs;
      if (it.out < base || it.out >= base + len) continue;
      auto &mp = it.integral ? imir : fmir;
      int &cells = it.integral ? icells : fcells;
      auto f = mp.find(base);
      if (f == mp.end()) {
        if (cells + len > 8 * 1024) return -1;
        mp[base] = cells;
        mirrors.push_back(DMirror{base, cells, (int)len, it.integral, 0});
        f = mp.find(base);
        cells += (int)len;
      }
      return f->second + (int)(it.out - base);
    }
    return -1;
  };
  std::vector<DEntry3> ent;
  for (const DCombItem &it : P.comb) {
    int og = og_of(it);
    if (og < 0) return false;  // an outer cell varies inside a block
    int so = mirror_of(it);
    int a = psi_a[it.psi], b = bpos[psi_b[it.psi]];
    if (it.integral && b >= nbi) return false;
    auto add = [&](int c, int yint, int64_t icell) {
      DEntry3 e{};
      e.a = a;
      e.b = b;
      e.c = c;
      e.yint = yint;
      e.integral = it.integral;
      e.og = og;
      e.so = so;
      e.out = it.out;
      e.cellmul = it.cellmul;
      e.icell = icell;
      ent.push_back(e);
    };
    if (it.block < 0) {
      add(it.col, it.integral ? 1 : 0, 0);  // B0: integral items read PHI0 integral columns
    } else {
      const DB1Set &S = P.b1sets[it.block];
      const auto &srefs = P.fast.b1[it.block].refs;
      for (int g = 0; g < S.G; ++g) {
        bool pick = true;
        for (int i = 0; i < S.nref; ++i)
          if (srefs[i].src == 4 && (g / S.radix[i]) % S.dom[i] != it.sel) pick = false;
        if (!pick) continue;
        int64_t ic = 0;
        for (int i = 0; i < S.nref; ++i) ic += ((g / S.radix[i]) % S.dom[i]) * P.grefs[it.ig0 + i].stride;
        int c = it.yint ? (int)(d.n0i + S.gbase_i + (int64_t)g * S.ni + it.col)
                        : (int)(d.n0f + S.gbase_f + (int64_t)g * S.nf + it.col);
        add(c, it.yint, ic);
      }
    }
  }
  std::vector<int> og_off{0};
  std::vector<DGroupRef> og_refs;
  for (auto &g : ogs) {
    og_refs.insert(og_refs.end(), g.begin(), g.end());
    og_off.push_back((int)og_refs.size());
  }
  d.nbst = (int)bstage.size();
  d.nbpart = (int)bpart.size();
  d.nb = (int)bdesc.size();
  d.nbi = nbi;
  d.nast = (int)astage.size();
  d.na = (int)adesc.size();
  d.nog = (int)ogs.size();
  d.nent = (int)ent.size();
  d.mirror_f = fcells;
  d.mirror_i = icells;
  d.nmirror = (int)mirrors.size();
  const bool c3_fits = combine3_smem(d, P.fp64) <= 222 * 1024;  // + static shared memory < 227 KB
  d.bstage = P.arena.upload(bstage.empty() ? std::vector<int2>{make_int2(0, 0)} : bstage, s);
  d.bterm = P.arena.upload(bdesc.empty() ? std::vector<DPsi>{DPsi{}} : bdesc, s);
  d.bpart = P.arena.upload(bpart.empty() ? std::vector<int>{0} : bpart, s);
  d.astage = P.arena.upload(astage.empty() ? std::vector<int2>{make_int2(0, 0)} : astage, s);
  d.aterm = P.arena.upload(adesc.empty() ? std::vector<DPsi>{DPsi{}} : adesc, s);
  d.apart = P.arena.upload(apart.empty() ? std::vector<int>{0} : apart, s);
  d.segfacs = P.arena.upload(sf2.empty() ? std::vector<DSegFac>{DSegFac{}} : sf2, s);
  d.og_off = P.arena.upload(og_off, s);
  d.grefs = P.arena.upload(og_refs.empty() ? std::vector<DGroupRef>{DGroupRef{}} : og_refs, s);
  d.ent = P.arena.upload(ent.empty() ? std::vector<DEntry3>{DEntry3{}} : ent, s);
  d.mirror = P.arena.upload(mirrors.empty() ? std::vector<DMirror>{DMirror{}} : mirrors, s);
  d.fsum = P.fsum;
  d.icnt = P.icnt;
  P.c3 = d;
  P.use_c5 = setup_combine5(ctx, P);
  if (!P.use_c5 && !c3_fits) return false;
  P.use_c3 = true;
  P.c3_block = 512;
  P.c3_grid = (int)std::max<int64_t>(1, std::min<int64_t>(148, d.nblocks));
  return true;
}

void setup_passes(lmfao_ctx *ctx, PhysPlan &P, const JoinTree &t) {
  cudaStream_t s = ctx->stream;
  // outputs and per-segment sums
  P.fsum = (double *)P.arena.alloc(std::max<int64_t>(1, P.nfsum) * 8);
  P.icnt = (unsigned long long *)P.arena.alloc(std::max<int64_t>(1, P.nicnt) * 8);
  size_t ts = P.fp64 ? 8 : 4;
  P.phi0f = P.arena.alloc(std::max<size_t>(1, P.nseg * P.b0f.size()) * ts);
  P.phi0i = (unsigned long long *)P.arena.alloc(std::max<size_t>(1, P.nseg * P.b0i.size()) * 8);
  P.wseg = (unsigned long long *)P.arena.alloc(P.nseg * 8);
  // segment decoding and outer view refs
  DSegment sg{};
  sg.ndig = (int)P.segcols.size();
  {
    int64_t acc = 1;
    for (int i = sg.ndig - 1; i >= 0; --i) { sg.radix[i] = acc; sg.dom[i] = P.segdom[i]; acc *= P.segdom[i]; }
  }
  std::vector<DOuter> outer;
  for (int c : P.outer) {
    const View &v = P.views[c];
    DOuter o{};
    o.v = view_ref(v);
    for (int d = 0; d < sg.ndig; ++d) {
      o.dstride[d] = 0;
      for (size_t i = 0; i < v.pkeycols.size(); ++i)
        if (v.pkeycols[i] == P.segcols[d]) o.dstride[d] = o.v.kstride[i];
    }
    outer.push_back(o);
  }
  // psi tables
  std::vector<DPsi> psi;
  std::vector<DSegFac> segfacs;
  std::vector<DPart> pparts;
  for (auto &p : P.psis) {
    DPsi d{};
    d.f0 = (int)segfacs.size();
    for (int f : p.segf) {
      const Fac &fc = P.facs[f];
      int dg = 0;
      for (size_t i = 0; i < P.segcols.size(); ++i) if (P.segcols[i] == fc.col) dg = (int)i;
      segfacs.push_back(DSegFac{dg, fc.pow, fc.ind, fc.op, fc.t});
    }
    d.nf = (int)p.segf.size();
    d.p0 = (int)pparts.size();
    for (auto &pp : p.parts) {
      const View &v = P.views[P.outer[pp.first]];
      // integral psi reads the exact FP64 value of an integral column
      pparts.push_back(DPart{pp.first, pp.second});
      (void)v;
    }
    d.np = (int)p.parts.size();
    d.integral = p.integral ? 1 : 0;
    psi.push_back(d);
  }
  // row tables
  std::vector<DMono> mono;
  std::vector<DFac> rfacs;
  for (auto &m : P.monos) {
    DMono d{(int)rfacs.size(), (int)m.size()};
    for (int f : m) {
      const Fac &fc = P.facs[f];
      rfacs.push_back(DFac{P.rowslot.at(fc.col), fc.ind, fc.pow, fc.op, fc.t});
    }
    mono.push_back(d);
  }
  std::vector<DRTerm> rts;
  std::vector<DPart> rparts;
  for (auto &r : P.rts) {
    DRTerm d{r.mono, (int)rparts.size(), (int)r.parts.size(), r.integral ? 1 : 0};
    for (auto &pp : r.parts) {
      const View &v = P.views[P.inner[pp.first]];
      int col = r.integral ? v.intcol[pp.second] : pp.second;
      if (col < 0) throw Error(LMFAO_ERR_ARG, "internal: integral term on a non-integral view column");
      rparts.push_back(DPart{pp.first, col});
    }
    rts.push_back(d);
  }
  std::vector<DViewRef> inner;
  for (int c : P.inner) {
    const View &v = P.views[c];
    DViewRef r = view_ref(v);
    for (int i = 0; i < r.nk; ++i) r.kcol[i] = P.rowslot.at(v.pkeycols[i]);
    inner.push_back(r);
  }
  // key columns of inner branches must be row slots (registered now if not yet)
  // segment weights
  DSegWeight sw{};
  sw.nseg = P.nseg;
  sw.seg = sg;
  sw.nouter = (int)outer.size();
  for (size_t i = 0; i < outer.size(); ++i) sw.outer[i] = outer[i];
  sw.wseg = P.wseg;
  P.sw = sw;
  // fact pass
  DFactPass &fp = P.fp;
  fp = DFactPass{};
  fp.nwork = P.nwork;
  fp.work = P.work;
  fp.wseg = P.wseg;
  fp.ncols = (int)P.rowdev.size();
  for (size_t i = 0; i < P.rowdev.size(); ++i) fp.col[i] = P.rowdev[i];
  fp.ninner = (int)inner.size();
  for (size_t i = 0; i < inner.size(); ++i) fp.inner[i] = inner[i];
  fp.nmono = (int)mono.size();
  fp.mono = P.arena.upload(mono, s);
  fp.facs = P.arena.upload(rfacs, s);
  fp.nrt = (int)rts.size();
  fp.rt = P.arena.upload(rts, s);
  fp.parts = P.arena.upload(rparts, s);
  fp.n0f = (int)P.b0f.size();
  fp.n0i = (int)P.b0i.size();
  fp.b0f = P.arena.upload(P.b0f, s);
  fp.b0i = P.arena.upload(P.b0i, s);
  fp.phi0f = P.phi0f;
  fp.phi0i = P.phi0i;
  fp.nb2 = (int)P.b2.size();
  fp.b2 = P.arena.upload(P.b2, s);
  fp.grefs = P.arena.upload(P.grefs, s);
  fp.thr = P.arena.upload(P.thr, s);
  fp.seg = sg;
  fp.nouter = (int)outer.size();
  for (size_t i = 0; i < outer.size(); ++i) fp.outer[i] = outer[i];
  fp.npsi = (int)psi.size();
  fp.psi = P.arena.upload(psi, s);
  fp.segfacs = P.arena.upload(segfacs, s);
  fp.psiparts = P.arena.upload(pparts, s);
  fp.fsum = P.fsum;
  fp.icnt = P.icnt;
  fp.b2_smem_items = std::max(1, (int)P.b2.size());
  P.nb0 = 4;
  while (P.nb0 < (int)P.b0f.size()) P.nb0 *= 2;
  if (P.nb0 > NB0_MAX) throw Error(LMFAO_ERR_UNSUPPORTED, "internal: too many per-segment sums");
  P.fp_block = 256;
  size_t fsm = fact_pass_smem(fp, P.fp64, P.fp_block);
  if (fsm > 200 * 1024) throw Error(LMFAO_ERR_UNSUPPORTED, "per-tuple items need more shared memory than available");
  int blocks_per_sm = 4;
  P.fp_grid = (int)std::max<int64_t>(1, std::min<int64_t>(148 * blocks_per_sm, (P.nwork + 7) / 8));
  // combine
  DCombine &cb = P.cb;
  cb = DCombine{};
  cb.nseg = P.nseg;
  cb.wseg = P.wseg;
  cb.seg = sg;
  cb.nouter = (int)outer.size();
  for (size_t i = 0; i < outer.size(); ++i) cb.outer[i] = outer[i];
  cb.npsi = (int)psi.size();
  cb.psi = fp.psi;
  cb.segfacs = fp.segfacs;
  cb.psiparts = fp.psiparts;
  cb.n0f = fp.n0f;
  cb.n0i = fp.n0i;
  cb.phi0f = P.phi0f;
  cb.phi0i = P.phi0i;
  cb.grefs = fp.grefs;
  cb.thr = fp.thr;
  cb.fsum = P.fsum;
  cb.icnt = P.icnt;
  if (P.fast.on) setup_fast(ctx, P, t, cb);
  setup_combine2(ctx, P, pparts);
  P.use_c3 = false;
  P.use_c4 = false;
  if (!P.no_c3) setup_combine3(ctx, P, psi, segfacs, pparts);
  if (!P.use_c3) setup_combine4(ctx, P, psi, segfacs, pparts);
  (void)t;
}

// Enqueue one evaluation of the batch on stream s.
void enqueue_run(lmfao_ctx *ctx, PhysPlan &P, const JoinTree &t, cudaStream_t s) {
  ctx->ev_names.clear();
  int ev = 0;
  auto mark = [&](const std::string &name) {
    if (!ctx->profiling) return;
    if ((int)ctx->events.size() <= ev) {
      cudaEvent_t e;
      LMFAO_CUDA(cudaEventCreate(&e));
      ctx->events.push_back(e);
    }
    LMFAO_CUDA(cudaEventRecord(ctx->events[ev++], s));
    ctx->ev_names.push_back(name);
  };
  mark("start");
  LMFAO_CUDA(cudaMemsetAsync(P.err, 0, 4, s));
  // views: the subtrees of different children of the root are independent, so (unless the run
  // is timed kernel by kernel) each runs on a side stream of its own, forked from and joined
  // back into s; within a subtree the post-order keeps children before parents. The zeroing of
  // the outputs and of the root pass's arrays runs on s meanwhile.
  std::vector<int> lane(P.vk.size(), -1);
  int nlanes = 0;
  if (!ctx->profiling && ctx->view_fork) {
    std::map<int, int> of_branch;
    for (size_t i = 0; i < P.vk.size(); ++i) {
      const int br = P.branch[P.vk_rel[i]];
      auto it = of_branch.find(br);
      if (it == of_branch.end()) it = of_branch.emplace(br, (int)(of_branch.size() % lmfao_ctx::kViewLanes)).first;
      lane[i] = it->second;
    }
    nlanes = std::min<int>((int)of_branch.size(), lmfao_ctx::kViewLanes);
    if (nlanes < 2) std::fill(lane.begin(), lane.end(), -1), nlanes = 0;
  }
  if (nlanes) {
    LMFAO_CUDA(cudaEventRecord(ctx->view_fork, s));
    for (int l = 0; l < nlanes; ++l) LMFAO_CUDA(cudaStreamWaitEvent(ctx->view_stream[l], ctx->view_fork, 0));
  }
  if (P.nfsum) LMFAO_CUDA(cudaMemsetAsync(P.fsum, 0, P.nfsum * 8, s));
  if (P.nicnt) LMFAO_CUDA(cudaMemsetAsync(P.icnt, 0, P.nicnt * 8, s));
  if (!P.fast.on && !P.b0f.empty()) LMFAO_CUDA(cudaMemsetAsync(P.phi0f, 0, P.nseg * P.b0f.size() * (P.fp64 ? 8 : 4), s));
  if (!P.fast.on && !P.b0i.empty()) LMFAO_CUDA(cudaMemsetAsync(P.phi0i, 0, P.nseg * P.b0i.size() * 8, s));
  if (P.fast.on) {
    const DFast &d = P.fd;
    if (d.nm * d.nw) LMFAO_CUDA(cudaMemsetAsync(P.phi0f, 0, P.nseg * d.nm * d.nw * (P.fp64 ? 8 : 4), s));
    if (d.n0i) LMFAO_CUDA(cudaMemsetAsync(P.phi0i, 0, P.nseg * d.n0i * 8, s));
    if (d.phi1f_seg) LMFAO_CUDA(cudaMemsetAsync(d.phi1f, 0, P.nseg * d.phi1f_seg * 4, s));
    if (d.phi1i_seg) LMFAO_CUDA(cudaMemsetAsync(d.phi1i, 0, P.nseg * d.phi1i_seg * 4, s));
    if (d.n3f) LMFAO_CUDA(cudaMemsetAsync(d.p3f, 0, d.nkeys * d.n3f * d.b3leaf * 8, s));
    if (d.n3f && !d.smem_p && !P.fp64) LMFAO_CUDA(cudaMemsetAsync(d.p3f32, 0, d.nkeys * d.n3f * d.b3leaf * 4, s));
    if (d.n3i) LMFAO_CUDA(cudaMemsetAsync(d.p3i, 0, d.nkeys * d.n3i * d.b3leaf * 8, s));
    LMFAO_CUDA(cudaMemsetAsync(d.ticket, 0, 4, s));
  }
  mark("memset");
  for (size_t i = 0; i < P.vk.size(); ++i) {
    int r = P.vk_rel[i];
    View &v = P.views[r];
    cudaStream_t vs = lane[i] >= 0 ? ctx->view_stream[lane[i]] : s;
    if (!v.keyrow) {  // the key-major kernel writes every cell
      LMFAO_CUDA(cudaMemsetAsync(v.v64, 0, v.nkeys * v.cols.size() * 8, vs));
      if (!v.codes.empty()) LMFAO_CUDA(cudaMemsetAsync(v.vcodes, 0xff, v.nkeys * v.codes.size() * 4, vs));
    }
    if (P.vgen[i].fn) LMFAO_CUDA(launch_gen_view(P.vgen[i], P.vk[i], vs));
    else launch_view_kernel(P.vk[i], vs);
    // the FP32 copy is read by the general fact pass only
    launch_view_finish(v.v64, P.fast.on ? nullptr : v.v32, v.vint, v.intcols_dev, (int)v.cols.size(), v.nint,
                       v.nkeys, P.err, vs);
    mark("view:" + ctx->rels[r].name);
  }
  for (int l = 0; l < nlanes; ++l) {
    LMFAO_CUDA(cudaEventRecord(ctx->view_join[l], ctx->view_stream[l]));
    LMFAO_CUDA(cudaStreamWaitEvent(s, ctx->view_join[l], 0));
  }
  launch_segment_weights(P.sw, s);
  mark("segment_weights");
  bool b3_side = false;
  if (P.fast.on) {
    const DFast &d = P.fd;
    if (d.ni) {
      const View &v = P.views[P.inner[0]];
      launch_fast_prep(d, v.v64, (int)v.cols.size(), P.fwcol_dev, v.vcodes, (int)v.codes.size(), P.fcodecol_dev,
                       const_cast<void *>(d.table), const_cast<int *>(d.codes), P.fp64, s, P.fibits_dev, P.fnibits);
    }
    if (P.gen.fn) {
      if (launch_gen_root_pass(P.gen, d, P.fast_grid, s) != cudaSuccess)
        throw Error(LMFAO_ERR_CUDA, "generated root pass: launch failed");
    } else if (!launch_fast_pass(d, P.fp64, P.fast_grid, P.fast_block, s)) {
      throw Error(LMFAO_ERR_UNSUPPORTED, "internal: no root-pass variant for this shape");
    }
    mark("fact_pass");
    if (P.b3f.nitems) {
      // the inner relation's outputs (atomic adds) are independent of the combine: on a side
      // stream, joined at the end of the run
      if (nlanes) {
        LMFAO_CUDA(cudaEventRecord(ctx->view_fork, s));
        LMFAO_CUDA(cudaStreamWaitEvent(ctx->view_stream[0], ctx->view_fork, 0));
        launch_b3_final(P.b3f, ctx->view_stream[0]);
        b3_side = true;
      } else {
        launch_b3_final(P.b3f, s);
      }
    }
    mark("b3_final");
  } else {
    launch_fact_pass(P.fp, P.fp64, P.nb0, P.fp_grid, P.fp_block, s);
    mark("fact_pass");
  }
  if (!P.comb.empty()) {
    if (P.use_c5) {
      launch_combine5_z(P.c5, P.fp64, s);
      mark("combine_z");
      launch_combine5_entries(P.c5, P.fp64, s);
    } else if (P.use_c3) launch_combine3(P.c3, P.fp64, P.c3_grid, P.c3_block, s);
    else if (P.use_c4) {
      const DComb4 &c4 = P.c4;
      if (c4.need_d0) {
        LMFAO_CUDA(cudaMemsetAsync(c4.yd0_f, 0, (size_t)c4.dom0 * c4.njobs * 8, s));
        LMFAO_CUDA(cudaMemsetAsync(c4.yd0_i, 0, (size_t)c4.dom0 * c4.njobs * 8, s));
      }
      if (c4.need_d1) {
        LMFAO_CUDA(cudaMemsetAsync(c4.yd1_f, 0, (size_t)c4.dom1 * c4.njobs * 8, s));
        LMFAO_CUDA(cudaMemsetAsync(c4.yd1_i, 0, (size_t)c4.dom1 * c4.njobs * 8, s));
      }
      LMFAO_CUDA(cudaMemsetAsync(c4.yall_f, 0, (size_t)c4.njobs * 8, s));
      LMFAO_CUDA(cudaMemsetAsync(c4.yall_i, 0, (size_t)c4.njobs * 8, s));
      launch_combine4(c4, P.fp64, s);
    } else {
      launch_combine2(P.c2, P.fp64, P.c2_grid, P.c2_block, s);
    }
  }
  mark("combine");
  if (b3_side) {
    LMFAO_CUDA(cudaEventRecord(ctx->view_join[0], ctx->view_stream[0]));
    LMFAO_CUDA(cudaStreamWaitEvent(s, ctx->view_join[0], 0));
  }
  LMFAO_CUDA(cudaGetLastError());
  (void)t;
}

// Bytes the fact pass must move per launch: the reorganised root columns it reads once,
// the work list, the segment weights, the inner views (read once; cache-resident after)
// and the per-segment sums it writes.
int64_t fact_pass_bytes(const lmfao_ctx *ctx, const PhysPlan &P) {
  const Relation &F = ctx->rels[P.root];
  int64_t b = 0;
  for (int c : P.rowcols) b += F.nrows * (F.cols[c].dtype == LMFAO_U8 ? 1 : 4);
  b += P.nwork * (int64_t)sizeof(DWork) + P.nseg * 8;
  int64_t ts = P.fp64 ? 8 : 4;
  for (int c : P.inner) {
    const View &v = P.views[c];
    b += v.nkeys * ((int64_t)v.cols.size() * ts + v.nint * 4 + (int64_t)v.codes.size() * 4);
  }
  b += P.nseg * ((int64_t)P.b0f.size() * ts + (int64_t)P.b0i.size() * 8);
  return b;
}

// Bytes the per-block contraction kernel must move per launch: the per-segment sums and segment
// weights it reads, the B-side view columns of every segment and the A-side ones of every
// block (FP64 views), and the Z, A and cell arrays it writes.
int64_t combine_z_bytes(const PhysPlan &P) {
  if (!P.use_c5) return 0;
  const DComb3 &d = P.c3;
  const int64_t ts = P.fp64 ? 8 : 4, nseg = d.nblocks * d.m, ny = d.nyf + d.nyi;
  int64_t b = nseg * ((int64_t)d.n0f * ts + d.phi1f_seg * 4 + (int64_t)d.n0i * 8 + d.phi1i_seg * 4 + 8);
  b += nseg * (int64_t)d.nbst * 8 + d.nblocks * (int64_t)d.nast * 8;
  b += d.nblocks * ((int64_t)d.nb * ny * ts + (int64_t)d.nbi * d.nyi * 8 + (int64_t)d.na * (ts + 8) + (int64_t)d.nog * 8);
  return b;
}
// Multiply-adds x 2 of the contraction Z_p = B_p^T Y_p over all blocks (the method's work; the
// split-BF16 form issues three such products on the tensor cores).
int64_t combine_z_flops(const PhysPlan &P) {
  if (!P.use_c5) return 0;
  const DComb3 &d = P.c3;
  return 2 * d.nblocks * d.m * (int64_t)d.nb * (d.nyf + d.nyi);
}

std::string json_escape(const std::string &x) {
  std::string o;
  for (char c : x) {
    if (c == '"' || c == '\\') o += '\\';
    o += c;
  }
  return o;
}

}  // namespace


// ======================================================================================
// plan building, candidates, features, cost model
// ======================================================================================
namespace {

constexpr int NFEAT = 32;

lmfao_plan_opts default_opts() {
  lmfao_plan_opts o{};
  o.precision = LMFAO_FP32;
  o.planner = LMFAO_PLAN_HEURISTIC;
  o.root_rel = -1;
  o.segment_rel = -2;
  o.mode = LMFAO_MODE_AUTO;
  return o;
}

// Options this engine does not evaluate are refused rather than replaced by others.
void check_plan_opts(const lmfao_ctx *ctx, const lmfao_plan_opts &o) {
  (void)ctx;
  if (o.precision != LMFAO_FP64 && o.precision != LMFAO_FP32 && o.precision != LMFAO_SPLIT_BF16)
    throw Error(LMFAO_ERR_ARG, "unknown precision " + std::to_string(o.precision));
  if (o.planner < LMFAO_PLAN_HEURISTIC || o.planner > LMFAO_PLAN_FORCED)
    throw Error(LMFAO_ERR_ARG, "unknown planner " + std::to_string(o.planner));
}

std::vector<int> parent_links(lmfao_ctx *ctx, const lmfao_plan_opts &o) {
  int n = (int)ctx->rels.size();
  std::vector<int> par;
  if (o.join_parent) {
    par.assign(o.join_parent, o.join_parent + n);
    for (int p : par)
      if (p < -1 || p >= n) throw Error(LMFAO_ERR_ARG, "join_parent out of range");
  } else if (n == 1) {
    par.assign(1, -1);
  } else {
    par = gyo(ctx);
  }
  return par;
}

int largest_relation(const lmfao_ctx *ctx) {
  int root = 0;
  for (int r = 1; r < (int)ctx->rels.size(); ++r)
    if (ctx->rels[r].nrows > ctx->rels[root].nrows) root = r;
  return root;
}

// Plan features of the learned cost model (sizes on a log10 scale).
std::vector<float> plan_features(const lmfao_ctx *ctx, const PhysPlan &P, const JoinTree &t) {
  auto lg = [](double x) { return (float)std::log10(1.0 + std::max(0.0, x)); };
  const double rows = (double)ctx->rels[P.root].nrows;
  double in_keys = 0, out_keys = 0, cols = 0, maxcols = 0, other_rows = 0;
  for (int c : P.inner) in_keys += (double)P.views[c].nkeys;
  for (int c : P.outer) out_keys += (double)P.views[c].nkeys;
  for (int r : t.post) {
    cols += (double)P.views[r].cols.size();
    maxcols = std::max(maxcols, (double)P.views[r].cols.size());
    other_rows += (double)ctx->rels[r].nrows;
  }
  double b0 = P.fast.on ? (double)(P.fast.monos.size() * P.fast.wcols.size()) : (double)(P.b0f.size() + P.b0i.size());
  double b1g = 0;
  for (auto &S : P.fast.b1) b1g += (double)S.G * (double)(S.fcols.size() + S.icols.size());
  double naggs = 0;
  for (auto &q : ctx->queries) naggs += (double)q.aggs.size();
  std::vector<float> f(NFEAT, 0.f);
  f[0] = lg(rows);
  f[1] = lg((double)P.nseg);
  f[2] = lg(rows / std::max<double>(1, (double)P.nseg));
  f[3] = (float)P.outer.size();
  f[4] = (float)P.inner.size();
  f[5] = lg(in_keys);
  f[6] = lg(out_keys);
  f[7] = lg(cols);
  f[8] = lg(maxcols);
  f[9] = lg(b0);
  f[10] = (float)P.fast.b1.size();
  f[11] = lg(b1g);
  f[12] = (float)P.fast.p3.size();
  f[13] = lg((double)P.b2.size());
  f[14] = lg((double)P.comb.size());
  f[15] = (P.prefix_len > 0 && !P.no_c3) ? 1.f : 0.f;
  f[16] = P.fast.on ? 1.f : 0.f;
  f[17] = (P.fast.on && P.fast.lean) ? 1.f : 0.f;
  f[18] = P.mode == LMFAO_MODE_GENERIC ? 1.f : 0.f;
  f[19] = lg((double)ctx->queries.size());
  f[20] = lg(naggs);
  f[21] = P.root == largest_relation(ctx) ? 1.f : 0.f;
  f[22] = lg(other_rows);
  f[23] = lg(rows * (1.0 + (double)P.inner.size()));
  // work estimates of the plan's kernels
  double rowbytes = 0;
  for (int c : P.rowcols) rowbytes += ctx->rels[P.root].cols[c].dtype == LMFAO_U8 ? 1 : 4;
  double b1cols = 0;
  for (auto &S : P.fast.b1) b1cols += (double)(S.fcols.size() + S.icols.size());
  double entries = 0;
  for (auto &c : P.comb) entries += c.block >= 0 && c.block < (int)P.fast.b1.size() ? (double)P.fast.b1[c.block].G : 1.0;
  double view_work = 0, inner_table = 0;
  for (int r : t.post) view_work += (double)ctx->rels[r].nrows * (double)P.views[r].cols.size();
  for (int c : P.inner) inner_table += (double)P.views[c].nkeys * (double)(P.fast.on ? P.fast.wcols.size() : P.views[c].cols.size());
  const double block = P.prefix_len > 0 ? std::max<double>(1, (double)P.nseg / (double)std::accumulate(
                                                P.segdom.begin(), P.segdom.begin() + P.prefix_len, int64_t(1),
                                                std::multiplies<int64_t>())) : 1.0;
  f[24] = lg(rows * rowbytes);
  f[25] = lg(rows * (b1cols + (double)P.fast.p3.size() + (double)P.fast.b4.size() + (double)P.b2.size()));
  f[26] = lg(entries * (double)P.nseg);
  f[27] = lg(entries * (double)P.nseg / block);
  f[28] = lg(view_work);
  f[29] = lg((double)P.nseg * (b0 + b1g));
  f[30] = lg(inner_table);
  f[31] = (float)(t.post.size() * 2 + 3);
  return f;
}

// Build the plan of options o into ctx (tree, logical plan, physical plan). With dry, stop
// after routing and return the plan features instead of setting up the device passes.
void build_plan(lmfao_ctx *ctx, const lmfao_plan_opts &o, bool dry, std::vector<float> *feats) {
  int n = (int)ctx->rels.size();
  std::vector<int> par = parent_links(ctx, o);
  int root = o.root_rel;
  if (root < 0 || root >= n || o.planner != LMFAO_PLAN_FORCED) {
    if (!(o.planner == LMFAO_PLAN_FORCED && root >= 0 && root < n)) root = largest_relation(ctx);
  }
  ctx->tree = build_tree(ctx, par, root);
  ctx->logical = build_logical(ctx, ctx->tree, o.query_root);
  if (ctx->device < 0) {  // host-only: the logical plan of Section 2 only
    ctx->planned = true;
    return;
  }
  PhysPlan *P = new PhysPlan();
  ctx->plan = P;
  P->fp64 = o.precision == LMFAO_FP64;
  P->split_bf16 = o.precision == LMFAO_SPLIT_BF16;
  P->no_c3 = o.combine == 1;
  P->mode = (o.mode == LMFAO_MODE_PER_TUPLE || o.mode == LMFAO_MODE_GENERIC) ? o.mode : LMFAO_MODE_FACTORISED;
  P->root = root;
  P->err = (int *)P->arena.alloc(16);
  Planner pl(ctx, *P, ctx->tree);
  pl.init_views();
  compute_multiplicities(ctx, *P, ctx->tree);
  pl.choose_segments(o);
  {
    bool done = false;
    if (P->mode == LMFAO_MODE_FACTORISED && pl.detect_family()) {
      pl.use_family = true;
      auto items = pl.decompose();
      done = pl.route_fast(items);
      if (!done) {  // filters go back to indicator factors
        pl.use_family = false;
        P->qout.clear();
      }
    }
    if (!done) {
      P->fast = PhysPlan::Fast{};
      P->comb.clear();
      auto items = pl.decompose();
      if (!(P->mode == LMFAO_MODE_FACTORISED && pl.route_fast(items))) {
        P->fast = PhysPlan::Fast{};
        P->comb.clear();
        pl.route_generic(items, P->mode);
      }
    }
  }
  for (int c : P->inner)
    for (int pc : P->views[c].pkeycols) pl.rowslot(pc);
  if (dry) {
    if (feats) *feats = plan_features(ctx, *P, ctx->tree);
    return;
  }
  setup_views(ctx, *P, ctx->tree, !P->fp64);
  setup_root(ctx, *P, ctx->tree);
  setup_passes(ctx, *P, ctx->tree);
  LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
  // side streams for views of different subtrees (once per context)
  if (!ctx->view_fork && P->vk.size() > 1) {
    LMFAO_CUDA(cudaEventCreateWithFlags(&ctx->view_fork, cudaEventDisableTiming));
    for (int i = 0; i < lmfao_ctx::kViewLanes; ++i) {
      LMFAO_CUDA(cudaStreamCreateWithFlags(&ctx->view_stream[i], cudaStreamNonBlocking));
      LMFAO_CUDA(cudaEventCreateWithFlags(&ctx->view_join[i], cudaEventDisableTiming));
    }
  }
  ctx->planned = true;
}

struct Cand {
  int root, seg, mode, combine;
};

// Candidate physical plans: root relation (the largest and the next two largest), segment
// relation (none or any child of the root), root pass (specialised when possible, or the
// generic pass) and combine (prefix-block or entry-wise).
std::vector<Cand> candidates(lmfao_ctx *ctx, const lmfao_plan_opts &o) {
  int n = (int)ctx->rels.size();
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctx->rels[a].nrows > ctx->rels[b].nrows; });
  std::vector<int> par = parent_links(ctx, o);
  std::vector<Cand> out;
  for (int ri = 0; ri < std::min(n, 3); ++ri) {
    int root = order[ri];
    JoinTree t = build_tree(ctx, par, root);
    std::vector<int> segs{-1};
    for (int c : t.children[root]) {
      int64_t nk = 1;
      for (auto &a : shared_attrs(ctx, c, root)) {
        nk *= ctx->rels[c].cols[ctx->rels[c].col(a)].domain;
        if (nk > (int64_t(1) << 26)) break;
      }
      if (nk <= (int64_t(1) << 26)) segs.push_back(c);
    }
    for (int sgi : segs)
      for (int mode : {LMFAO_MODE_AUTO, LMFAO_MODE_GENERIC})
        for (int comb : {0, 1}) {
          if (mode == LMFAO_MODE_GENERIC && comb == 1) continue;
          out.push_back(Cand{root, sgi, mode, comb});
        }
  }
  return out;
}

lmfao_plan_opts cand_opts(const lmfao_plan_opts &base, const Cand &c) {
  lmfao_plan_opts o = base;
  o.planner = LMFAO_PLAN_FORCED;
  o.root_rel = c.root;
  o.segment_rel = c.seg;
  o.mode = c.mode;
  o.combine = c.combine;
  return o;
}

// Median device time of `reps` evaluations of the current plan after `warm` warm-up runs.
double time_plan(lmfao_ctx *ctx, int warm, int reps) {
  PhysPlan &P = *ctx->plan;
  cudaStream_t s = ctx->stream;
  for (int i = 0; i < warm; ++i) enqueue_run(ctx, P, ctx->tree, s);
  cudaEvent_t a, b;
  LMFAO_CUDA(cudaEventCreate(&a));
  LMFAO_CUDA(cudaEventCreate(&b));
  std::vector<double> ms;
  for (int i = 0; i < reps; ++i) {
    LMFAO_CUDA(cudaEventRecord(a, s));
    enqueue_run(ctx, P, ctx->tree, s);
    LMFAO_CUDA(cudaEventRecord(b, s));
    LMFAO_CUDA(cudaEventSynchronize(b));
    float f = 0;
    LMFAO_CUDA(cudaEventElapsedTime(&f, a, b));
    ms.push_back(f);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  std::sort(ms.begin(), ms.end());
  return ms[ms.size() / 2];
}

// ------------------------------------------------------------------ tile autotuner
// Launch shapes that change speed but not results: the root pass's work-item length (tuples
// per work item taken from the ticket) and the per-block combine's chunk of segments. The
// tuner times whole runs of the plan on its data for a small candidate set (coordinate search:
// work-item length first, then the chunk), keeps the fastest and records it in a cache file
// (LMFAO_TUNE_CACHE, default ~/.cache/lmfao/tiles.txt) under a key of the plan's shape and the
// device, so a later plan of the same shape takes the tiles without timing.

void set_work_chunk(lmfao_ctx *ctx, PhysPlan &P, int chunk) {
  if (P.seg_hist.empty()) return;
  P.work_chunk = chunk;
  build_work(ctx, P);
  P.fd.nwork = P.nwork;
  P.fd.work = P.work;
  P.fd.work_q = P.work_q;
  P.fp.nwork = P.nwork;
  P.fp.work = P.work;
  if (P.gen.fn) {
    int per_sm = 1, nsm = 148;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.gen.fn, P.gen.block, P.gen.smem);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    cudaGetLastError();
    P.fast_grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(1, per_sm), P.nwork));
  }
}

// Lane layout of the generated lean root pass (one tuple per lane, or a 4-tuple quad per lane);
// regenerates (or takes from the process cache) the kernel. False when not applicable.
bool set_root_lanes(lmfao_ctx *ctx, PhysPlan &P, int lanes) {
  if (!P.gen.fn || P.gen.family || !P.fd.lean) return false;
  DFast d = P.fd;
  d.lanes = lanes;
  GenRootPass g = gen_root_pass(d, P.fp64, ctx->device, P.thr);
  if (!g.fn) return false;
  P.fd.lanes = lanes;
  P.gen = g;
  int per_sm = 1, nsm = 148;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, P.gen.fn, P.gen.block, P.gen.smem);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  cudaGetLastError();
  P.fast_grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)nsm * std::max(1, per_sm), P.nwork));
  return true;
}

// A chunk of segments for the two-kernel block combine: a multiple of 16 on the tensor-core
// path; rejected when its tables do not fit shared memory or break the bulk-copy alignment.
bool set_combine_chunk(PhysPlan &P, int kc) {
  if (!P.use_c5) return false;
  DComb5 D = P.c5;
  const int64_t m = D.c.m;
  if (D.tc) kc = (int)std::min<int64_t>(kc, (m + 15) / 16 * 16);
  else kc = (int)std::min<int64_t>(kc, m);
  if (kc < 1 || (D.tc && kc % 16)) return false;
  D.kc = kc;
  if (combine5_smem(D, P.fp64) > 200 * 1024) return false;
  if (D.bulk) {
    const int64_t ts = P.fp64 ? 8 : 4;
    const int64_t rb[5] = {(int64_t)D.c.n0f * ts, D.c.phi1f_seg * 4, (int64_t)D.c.n0i * 8, D.c.phi1i_seg * 4, 8};
    for (int i = 0; i < 5; ++i)
      if (rb[i] && ((int64_t)kc * rb[i]) % 16) return false;
  }
  P.c5 = D;
  return true;
}

std::string tune_key(const lmfao_ctx *ctx, const PhysPlan &P) {
  std::ostringstream k;
  cudaDeviceProp pr{};
  cudaGetDeviceProperties(&pr, ctx->device);
  std::string name = pr.name;
  for (char &c : name)
    if (c == ' ') c = '_';
  k << name << "/" << pr.multiProcessorCount << "/" << (P.fp64 ? "fp64" : P.split_bf16 ? "bf16x3" : "fp32") << "/"
    << ctx->rels[P.root].nrows << "/" << P.nseg << "/" << P.gen.source_hash << "/" << P.use_c5 << "/" << P.c3.nb
    << "x" << P.c3.nyf + P.c3.nyi << "x" << P.c3.m << "x" << P.c3.nblocks << "/" << P.c3.nent;
  return k.str();
}

std::string tune_cache_path() {
  if (const char *p = std::getenv("LMFAO_TUNE_CACHE")) return p;
  const char *home = std::getenv("HOME");
  return std::string(home ? home : "/tmp") + "/.cache/lmfao/tiles.txt";
}

void autotune(lmfao_ctx *ctx, PhysPlan &P) {
  const auto t0 = std::chrono::steady_clock::now();
  const std::string key = tune_key(ctx, P), path = tune_cache_path();
  P.tuned = true;
  {
    std::ifstream in(path);
    std::string k;
    int wc = 0, kc = 0, ln = -1;
    double ms = 0;
    while (in >> k >> wc >> kc >> ln >> ms)
      if (k == key) {
        if (ln >= 0 && ln != P.fd.lanes) set_root_lanes(ctx, P, ln);
        if (wc > 0) set_work_chunk(ctx, P, wc);
        if (kc > 0) set_combine_chunk(P, kc);
        P.tune_cached = true;
      }
    if (P.tune_cached) {
      P.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      return;
    }
  }
  double best = time_plan(ctx, 1, 3);
  P.tune_candidates = 1;
  int best_ln = P.fd.lanes;
  if (set_root_lanes(ctx, P, 1 - best_ln)) {
    const double ms = time_plan(ctx, 1, 3);
    ++P.tune_candidates;
    if (ms < best) { best = ms; best_ln = 1 - best_ln; }
    else set_root_lanes(ctx, P, best_ln);
  }
  int best_wc = P.work_chunk;
  if (!P.seg_hist.empty()) {
    for (int wc : {1024, 2048, 8192, 16384}) {
      set_work_chunk(ctx, P, wc);
      const double ms = time_plan(ctx, 1, 3);
      ++P.tune_candidates;
      if (ms < best) { best = ms; best_wc = wc; }
    }
    set_work_chunk(ctx, P, best_wc);
  }
  int best_kc = P.use_c5 ? P.c5.kc : 0;
  if (P.use_c5) {
    for (int kc : {16, 32, 64, 128}) {
      if (kc == best_kc || !set_combine_chunk(P, kc)) continue;
      const double ms = time_plan(ctx, 1, 3);
      ++P.tune_candidates;
      if (ms < best) { best = ms; best_kc = kc; }
    }
    set_combine_chunk(P, best_kc);
  }
  // append the winner to the cache file (one line per key; the last line of a key wins)
  const std::string dir = path.substr(0, path.find_last_of('/'));
  if (!dir.empty()) {
    for (size_t i = 1; i <= dir.size(); ++i)
      if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
  }
  std::ofstream out(path, std::ios::app);
  if (out) out << key << " " << best_wc << " " << best_kc << " " << (P.gen.fn && !P.gen.family ? best_ln : -1) << " "
                << best << "\n";
  P.tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Whether the last evaluation of the current plan passed its device checks (group-by
// attributes determined by the join keys of their relations, exact 32-bit view counts).
// A plan whose checks fail on the loaded data cannot be chosen by a planner.
// Runs the view kernels of the current plan once on the context's stream and returns the
// device error flags they raise (1: a group-by attribute of a non-root relation is not
// determined by the key of that relation's view toward the root; 2: a count above 2^32).
int view_flags(lmfao_ctx *ctx) {
  PhysPlan &P = *ctx->plan;
  cudaStream_t s = ctx->stream;
  LMFAO_CUDA(cudaMemsetAsync(P.err, 0, 4, s));
  for (size_t i = 0; i < P.vk.size(); ++i) {
    View &v = P.views[P.vk_rel[i]];
    if (!v.keyrow) {
      LMFAO_CUDA(cudaMemsetAsync(v.v64, 0, v.nkeys * v.cols.size() * 8, s));
      if (!v.codes.empty()) LMFAO_CUDA(cudaMemsetAsync(v.vcodes, 0xff, v.nkeys * v.codes.size() * 4, s));
    }
    if (P.vgen[i].fn) LMFAO_CUDA(launch_gen_view(P.vgen[i], P.vk[i], s));
    else launch_view_kernel(P.vk[i], s);
    launch_view_finish(v.v64, v.v32, v.vint, v.intcols_dev, (int)v.cols.size(), v.nint, v.nkeys, P.err, s);
  }
  LMFAO_CUDA(cudaGetLastError());
  int e = 0;
  LMFAO_CUDA(cudaStreamSynchronize(s));
  LMFAO_CUDA(cudaMemcpy(&e, P.err, 4, cudaMemcpyDeviceToHost));
  return e;
}

bool views_carry_codes(const PhysPlan &P) {
  for (size_t i = 0; i < P.vk.size(); ++i)
    if (!P.views[P.vk_rel[i]].codes.empty()) return true;
  return false;
}

bool plan_checks_pass(lmfao_ctx *ctx) {
  int e = 0;
  LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
  LMFAO_CUDA(cudaMemcpy(&e, ctx->plan->err, 4, cudaMemcpyDeviceToHost));
  return e == 0;
}

struct CostModelFile {
  int d = 0, nmodels = 1;
  std::vector<float> mean, std;
  std::vector<std::vector<float>> params;  // one parameter vector per ensemble member
};

// Text file: "lmfao-cost-model 2 <d> <nmodels>", then d feature means, d standard
// deviations, then nmodels x lmfao_mlp_param_count(d) parameters (whitespace separated).
// The prediction is the mean over the ensemble.
CostModelFile load_cost_model(const char *path) {
  if (!path) throw Error(LMFAO_ERR_ARG, "the learned planner needs a cost model file");
  FILE *f = std::fopen(path, "r");
  if (!f) throw Error(LMFAO_ERR_ARG, std::string("cannot open cost model ") + path);
  CostModelFile cm;
  char tag[64] = {0};
  int ver = 0;
  bool ok = std::fscanf(f, "%63s %d %d %d", tag, &ver, &cm.d, &cm.nmodels) == 4 &&
            std::string(tag) == "lmfao-cost-model" && ver == 2 && cm.d == NFEAT && cm.nmodels >= 1 &&
            cm.nmodels <= 64;
  int64_t np = ok ? mlp_param_count(cm.d) : 0;
  auto rd = [&](std::vector<float> &v, int64_t k) {
    v.resize(k);
    for (int64_t i = 0; i < k && ok; ++i) ok = std::fscanf(f, "%f", &v[i]) == 1;
  };
  if (ok) rd(cm.mean, cm.d);
  if (ok) rd(cm.std, cm.d);
  cm.params.resize(ok ? cm.nmodels : 0);
  for (int m = 0; m < cm.nmodels && ok; ++m) rd(cm.params[m], np);
  std::fclose(f);
  if (!ok) throw Error(LMFAO_ERR_ARG, std::string("malformed cost model ") + path);
  for (float &x : cm.std)
    if (!(x > 0)) x = 1.f;
  return cm;
}

std::vector<float> predict(const CostModelFile &cm, const std::vector<float> &X, int n) {
  float *dx = nullptr, *dp = nullptr, *dy = nullptr;
  LMFAO_CUDA(cudaMalloc(&dx, X.size() * 4 + 16));
  LMFAO_CUDA(cudaMalloc(&dp, cm.params[0].size() * 4 + 16));
  LMFAO_CUDA(cudaMalloc(&dy, (size_t)n * 4 + 16));
  LMFAO_CUDA(cudaMemcpy(dx, X.data(), X.size() * 4, cudaMemcpyHostToDevice));
  std::vector<float> y(n, 0.f), ym(n);
  int rc = LMFAO_OK;
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < cm.nmodels && rc == LMFAO_OK && e == cudaSuccess; ++m) {
    e = cudaMemcpy(dp, cm.params[m].data(), cm.params[m].size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) rc = lmfao_mlp_forward(dx, n, cm.d, dp, nullptr, nullptr, dy, nullptr);
    if (rc == LMFAO_OK && e == cudaSuccess) e = cudaMemcpy(ym.data(), dy, (size_t)n * 4, cudaMemcpyDeviceToHost);
    for (int i = 0; i < n; ++i) y[i] += ym[i] / cm.nmodels;
  }
  cudaFree(dx);
  cudaFree(dp);
  cudaFree(dy);
  if (rc != LMFAO_OK || e != cudaSuccess) throw Error(LMFAO_ERR_CUDA, "cost model evaluation failed");
  return y;
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
namespace lmfao {

// SUM(y) has one factor y (or y^1); SUM(y^2) has y^2 or y * y. Returns the attribute in *attr
// and the power (1 or 2), or 0 when the aggregate is neither.
static int single_attr_power(const std::vector<FactorIn> &fs, std::string *attr) {
  int pw = 0;
  for (const FactorIn &f : fs) {
    if (!attr->empty() && f.attr != *attr) return 0;
    *attr = f.attr;
    pw += f.fn == LMFAO_FN_POW ? f.param : 1;
  }
  return fs.empty() ? 0 : pw;
}

int cart_descriptors(lmfao_ctx *ctx, const int *qids, int n, int64_t *desc, PhysPlan **plan) {
  if (!ctx->ran || (!ctx->plan && ctx->subs.empty())) throw Error(LMFAO_ERR_NOT_PLANNED, "no run yet");
  PhysPlan *PP = nullptr;
  int nb = 0;
  for (int i = 0; i < n; ++i) {
    const int q0 = qids[i];
    if (q0 < 0 || q0 >= (int)ctx->queries.size()) throw Error(LMFAO_ERR_ARG, "bad query id " + std::to_string(q0));
    const auto pq = plan_of(ctx, q0);
    if (PP && pq.first != PP)
      throw Error(LMFAO_ERR_UNSUPPORTED, "the queries are evaluated by plans with different roots");
    PP = pq.first;
    const PhysPlan &P = *PP;
    const int q = q0;
    const QueryIn &Q = ctx->queries[q];
    const char *shape = "CART variances need one BUCKET group-by and aggregates COUNT, SUM(y), SUM(y^2) of one "
                        "attribute y (in any order)";
    if (Q.gb.size() != 1 || Q.gb[0].kind != LMFAO_GB_BUCKET || Q.aggs.size() != 3)
      throw Error(LMFAO_ERR_ARG, std::string(shape) + " (query " + std::to_string(q) + ")");
    int ic = -1, i1 = -1, i2 = -1;
    std::string y;
    for (int a = 0; a < 3; ++a) {
      std::string attr = y;
      const int pw = Q.aggs[a].empty() ? -1 : single_attr_power(Q.aggs[a], &attr);
      if (pw == -1 && ic < 0) ic = a;
      else if (pw == 1 && i1 < 0) { i1 = a; y = attr; }
      else if (pw == 2 && i2 < 0) { i2 = a; y = attr; }
      else throw Error(LMFAO_ERR_ARG, std::string(shape) + " (query " + std::to_string(q) + ")");
    }
    const QueryOut &qo = P.qout[pq.second];
    if (qo.integral[i1] || qo.integral[i2])
      throw Error(LMFAO_ERR_ARG, std::string(shape) + ": y must be a value attribute (query " + std::to_string(q) + ")");
    const int b = (int)Q.gb[0].thr.size() + 1;
    if (i && b != nb) throw Error(LMFAO_ERR_ARG, "all queries need the same number of buckets");
    nb = b;
    if ((int)qo.cells != nb) throw Error(LMFAO_ERR_ARG, "all queries need the same number of buckets");
    if (desc) {
      int64_t *d = desc + (size_t)i * kCartDescWords;
      d[0] = qo.io;
      d[1] = qo.fo;
      d[2] = qo.cells;
      d[3] = qo.naggs;
      d[4] = i1;
      d[5] = i2;
    }
  }
  if (plan) *plan = PP ? PP : ctx->plan;
  return nb;
}

}  // namespace lmfao

extern "C" {

int lmfao_create(lmfao_ctx **out, int device) {
  if (!out) return LMFAO_ERR_ARG;
  *out = nullptr;
  if (device == -1) {  // host-only context: schema, batch and logical plan, no device work
    lmfao_ctx *ctx = new lmfao_ctx();
    ctx->device = -1;
    *out = ctx;
    return LMFAO_OK;
  }
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return LMFAO_ERR_CUDA;
  }
  lmfao_ctx *ctx = new lmfao_ctx();
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess || cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return LMFAO_ERR_CUDA;
  }
  *out = ctx;
  return LMFAO_OK;
}

int lmfao_destroy(lmfao_ctx *ctx) {
  if (!ctx) return LMFAO_ERR_ARG;
  if (ctx->device >= 0) cudaSetDevice(ctx->device);
  drop_plan(ctx);
  for (auto &R : ctx->rels)
    for (auto &c : R.cols)
      if (c.owned && c.dev) cudaFree(c.dev);
  for (auto &E : ctx->reorg) {
    if (E.dest) cudaFree(E.dest);
    for (auto &kv : E.cols) cudaFree(kv.second);
  }
  for (auto e : ctx->events) cudaEventDestroy(e);
  for (int i = 0; i < lmfao_ctx::kViewLanes; ++i) {
    if (ctx->view_stream[i]) cudaStreamDestroy(ctx->view_stream[i]);
    if (ctx->view_join[i]) cudaEventDestroy(ctx->view_join[i]);
  }
  if (ctx->view_fork) cudaEventDestroy(ctx->view_fork);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return LMFAO_OK;
}

const char *lmfao_last_error(const lmfao_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int lmfao_load_relation(lmfao_ctx *ctx, const char *name, int64_t nrows, const lmfao_column *cols, int ncols,
                        uint32_t flags, int *rel_id) {
  return guarded(ctx, [&]() -> int {
    if (!name || nrows < 0 || (ncols > 0 && !cols) || ncols <= 0 || flags > LMFAO_ADOPT_DEVICE)
      return fail(ctx, LMFAO_ERR_ARG, "bad relation arguments");
    if (nrows > (int64_t(1) << 31) - 1) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "relations are limited to 2^31-1 tuples");
    for (auto &R : ctx->rels)
      if (R.name == name) return fail(ctx, LMFAO_ERR_ARG, std::string("relation ") + name + " already loaded");
    Relation R;
    R.name = name;
    R.nrows = nrows;
    for (int i = 0; i < ncols; ++i) {
      const lmfao_column &c = cols[i];
      if (!c.attr || (!c.data && nrows > 0)) return fail(ctx, LMFAO_ERR_ARG, "column without name or data");
      for (auto &o : R.cols)
        if (o.attr == c.attr) return fail(ctx, LMFAO_ERR_ARG, std::string("duplicate attribute ") + c.attr);
      if (c.role < LMFAO_KEY || c.role > LMFAO_CONT) return fail(ctx, LMFAO_ERR_ARG, "bad column role");
      bool ok = (c.role == LMFAO_CONT) ? (c.dtype == LMFAO_F32 || c.dtype == LMFAO_U8) : c.dtype == LMFAO_I32;
      if (!ok) return fail(ctx, LMFAO_ERR_DTYPE, std::string("dtype not allowed for column ") + c.attr);
      if (c.role != LMFAO_CONT && (c.domain <= 0 || c.domain > (int64_t(1) << 31)))
        return fail(ctx, LMFAO_ERR_ARG, std::string("column ") + c.attr + " needs a domain in [1, 2^31]");
    }
    if (ctx->device < 0) {  // host-only: keep the schema and cardinalities, validate keys
      if (flags != LMFAO_HOST) return fail(ctx, LMFAO_ERR_ARG, "a host-only context takes host columns");
      for (int i = 0; i < ncols; ++i) {
        const lmfao_column &c = cols[i];
        if (c.role != LMFAO_CONT) {
          const int32_t *v = (const int32_t *)c.data;
          for (int64_t r = 0; r < nrows; ++r)
            if (v[r] < 0 || v[r] >= c.domain)
              return fail(ctx, LMFAO_ERR_KEY_RANGE, std::string("value of ") + c.attr + " outside its domain");
        }
        Column col;
        col.attr = c.attr;
        col.dtype = c.dtype;
        col.role = c.role;
        col.domain = c.domain;
        R.cols.push_back(col);
      }
      drop_plan(ctx);
      ctx->rels.push_back(R);
      if (rel_id) *rel_id = (int)ctx->rels.size() - 1;
      return LMFAO_OK;
    }
    std::vector<void *> mine;
    try {
      for (int i = 0; i < ncols; ++i) {
        const lmfao_column &c = cols[i];
        Column col;
        col.attr = c.attr;
        col.dtype = c.dtype;
        col.role = c.role;
        col.domain = c.domain;
        size_t esz = c.dtype == LMFAO_U8 ? 1 : 4;
        if (c.role != LMFAO_CONT && flags == LMFAO_HOST) {
          const int32_t *v = (const int32_t *)c.data;
          for (int64_t r = 0; r < nrows; ++r)
            if (v[r] < 0 || v[r] >= c.domain)
              throw Error(LMFAO_ERR_KEY_RANGE, std::string("value ") + std::to_string(v[r]) + " of " + c.attr +
                                                   " outside [0, " + std::to_string(c.domain) + ")");
        }
        if (flags == LMFAO_ADOPT_DEVICE) {
          col.dev = const_cast<void *>(c.data);
          col.owned = false;
        } else {
          LMFAO_CUDA(cudaMalloc(&col.dev, std::max<size_t>(16, nrows * esz)));
          mine.push_back(col.dev);
          col.owned = true;
          if (nrows)
            LMFAO_CUDA(cudaMemcpyAsync(col.dev, c.data, nrows * esz,
                                       flags == LMFAO_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                       ctx->stream));
        }
        if (c.role != LMFAO_CONT && flags != LMFAO_HOST && nrows) {
          int *bad = nullptr;
          LMFAO_CUDA(cudaMalloc(&bad, 4));
          mine.push_back(bad);
          LMFAO_CUDA(cudaMemsetAsync(bad, 0, 4, ctx->stream));
          launch_range_check(col.dev, c.dtype, nrows, c.domain, bad, ctx->stream);
          int hb = 0;
          LMFAO_CUDA(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, ctx->stream));
          LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
          cudaFree(bad);
          mine.pop_back();
          if (hb) throw Error(LMFAO_ERR_KEY_RANGE, std::string("a value of ") + c.attr + " lies outside its domain");
        }
        R.cols.push_back(col);
      }
      LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
      for (void *p : mine) cudaFree(p);
      throw;
    }
    drop_plan(ctx);
    ctx->rels.push_back(R);
    if (rel_id) *rel_id = (int)ctx->rels.size() - 1;
    return LMFAO_OK;
  });
}

int lmfao_add_batch(lmfao_ctx *ctx, const lmfao_aggregate *aggs, int naggs, const lmfao_groupby *gb, int ngb,
                    const lmfao_predicate *filters, int nfilters, int *query_id) {
  return guarded(ctx, [&]() -> int {
    if (naggs < 0 || ngb < 0 || nfilters < 0 || (naggs && !aggs) || (ngb && !gb) || (nfilters && !filters))
      return fail(ctx, LMFAO_ERR_ARG, "bad batch arguments");
    auto find_attr = [&](const char *a) -> const Column * {
      if (!a) return nullptr;
      for (auto &R : ctx->rels) {
        int c = R.col(a);
        if (c >= 0) return &R.cols[c];
      }
      return nullptr;
    };
    QueryIn q;
    for (int i = 0; i < naggs; ++i) {
      std::vector<FactorIn> fs;
      if (aggs[i].nfactors < 0 || (aggs[i].nfactors && !aggs[i].factors)) return fail(ctx, LMFAO_ERR_ARG, "bad aggregate");
      for (int j = 0; j < aggs[i].nfactors; ++j) {
        const lmfao_factor &f = aggs[i].factors[j];
        if (!find_attr(f.attr)) return fail(ctx, LMFAO_ERR_ARG, std::string("unknown attribute ") + (f.attr ? f.attr : "(null)"));
        if (f.fn != LMFAO_FN_ID && f.fn != LMFAO_FN_POW) return fail(ctx, LMFAO_ERR_ARG, "unknown factor function");
        if (f.fn == LMFAO_FN_POW && (f.param < 1 || f.param > 16)) return fail(ctx, LMFAO_ERR_ARG, "POW exponent must be in [1, 16]");
        fs.push_back(FactorIn{f.attr, f.fn, f.fn == LMFAO_FN_POW ? f.param : 1});
      }
      q.aggs.push_back(fs);
    }
    for (int i = 0; i < ngb; ++i) {
      const Column *c = find_attr(gb[i].attr);
      if (!c) return fail(ctx, LMFAO_ERR_ARG, std::string("unknown group-by attribute ") + (gb[i].attr ? gb[i].attr : "(null)"));
      GroupIn g{gb[i].attr, gb[i].kind, {}};
      if (g.kind == LMFAO_GB_VALUE) {
        if (c->role == LMFAO_CONT) return fail(ctx, LMFAO_ERR_ARG, "VALUE group-by needs a KEY or CAT attribute");
      } else if (g.kind == LMFAO_GB_BUCKET) {
        if (gb[i].nthresholds < 0 || (gb[i].nthresholds && !gb[i].thresholds)) return fail(ctx, LMFAO_ERR_ARG, "bad thresholds");
        g.thr.assign(gb[i].thresholds, gb[i].thresholds + gb[i].nthresholds);
        for (size_t k = 1; k < g.thr.size(); ++k)
          if (!(g.thr[k - 1] < g.thr[k])) return fail(ctx, LMFAO_ERR_ARG, "thresholds must be strictly ascending");
      } else return fail(ctx, LMFAO_ERR_ARG, "unknown group-by kind");
      for (auto &o : q.gb) if (o.attr == g.attr && o.kind == g.kind && o.thr == g.thr) return fail(ctx, LMFAO_ERR_ARG, "repeated group-by");
      q.gb.push_back(g);
    }
    for (int i = 0; i < nfilters; ++i) {
      if (!find_attr(filters[i].attr)) return fail(ctx, LMFAO_ERR_ARG, std::string("unknown filter attribute ") + (filters[i].attr ? filters[i].attr : "(null)"));
      if (filters[i].op < LMFAO_LE || filters[i].op > LMFAO_NE) return fail(ctx, LMFAO_ERR_ARG, "unknown predicate");
      q.filters.push_back(PredIn{filters[i].attr, filters[i].op, filters[i].t});
    }
    drop_plan(ctx);
    ctx->queries.push_back(q);
    if (query_id) *query_id = (int)ctx->queries.size() - 1;
    return LMFAO_OK;
  });
}

int lmfao_clear_batch(lmfao_ctx *ctx) {
  return guarded(ctx, [&]() -> int {
    drop_plan(ctx);
    ctx->queries.clear();
    return LMFAO_OK;
  });
}

int lmfao_plan(lmfao_ctx *ctx, const lmfao_plan_opts *opts, lmfao_plan_info *info) {
  return guarded(ctx, [&]() -> int {
    auto t0 = std::chrono::steady_clock::now();
    drop_plan(ctx);
    if (ctx->rels.empty()) return fail(ctx, LMFAO_ERR_ARG, "no relations loaded");
    lmfao_plan_opts o = default_opts();
    if (opts) o = *opts;
    check_plan_opts(ctx, o);
    double predicted = -1;
    if (ctx->device >= 0 && (o.planner == LMFAO_PLAN_EXHAUSTIVE || o.planner == LMFAO_PLAN_LEARNED)) {
      std::vector<Cand> cands = candidates(ctx, o);
      if (cands.empty()) return fail(ctx, LMFAO_ERR_ARG, "no candidate plan");
      int best = -1;
      if (o.planner == LMFAO_PLAN_EXHAUSTIVE) {
        double bt = 1e300;
        for (size_t c = 0; c < cands.size(); ++c) {
          build_plan(ctx, cand_opts(o, cands[c]), false, nullptr);
          double ms = time_plan(ctx, 1, 3);
          const bool ok = plan_checks_pass(ctx);
          drop_plan(ctx);
          if (ok && ms < bt) { bt = ms; best = (int)c; }
        }
        if (best < 0) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "no candidate plan passes its checks on this data");
        predicted = bt;
      } else {
        CostModelFile cm = load_cost_model(o.cost_model);
        std::vector<float> X;
        for (auto &c : cands) {
          std::vector<float> f;
          build_plan(ctx, cand_opts(o, c), true, &f);
          drop_plan(ctx);
          for (size_t k = 0; k < f.size(); ++k) X.push_back((f[k] - cm.mean[k]) / cm.std[k]);
        }
        std::vector<float> y = predict(cm, X, (int)cands.size());
        // the candidate of least predicted time among those that pass their checks
        std::vector<int> order(cands.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return y[a] < y[b]; });
        // the model ranks; the first learned_topk candidates that pass their checks are timed
        // (one of them only: no timing) and the fastest is kept
        const int topk = std::max(1, o.learned_topk);
        double bt = 1e300;
        int measured = 0;
        for (int c : order) {
          build_plan(ctx, cand_opts(o, cands[c]), false, nullptr);
          const double ms = topk > 1 ? time_plan(ctx, 1, 3) : (enqueue_run(ctx, *ctx->plan, ctx->tree, ctx->stream), 0.0);
          const bool ok = plan_checks_pass(ctx);
          drop_plan(ctx);
          if (!ok) continue;
          if (ms < bt) { bt = ms; best = c; }
          if (++measured >= topk) break;
        }
        if (best < 0) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "no candidate plan passes its checks on this data");
        predicted = std::exp((double)y[best]);
      }
      build_plan(ctx, cand_opts(o, cands[best]), false, nullptr);
    } else {
      build_plan(ctx, o, false, nullptr);
      // A group-by attribute of a non-root relation must be determined by the key of that
      // relation's view toward the root (checked on the loaded data by the view kernels). The
      // heuristic planner then tries the other relations as root, largest first; a forced root
      // that fails is an error of the plan.
      if (ctx->device >= 0 && ctx->plan && views_carry_codes(*ctx->plan) && (view_flags(ctx) & 1)) {
        const int bad_root = ctx->plan->root;
        drop_plan(ctx);
        const std::string msg = "a group-by attribute of a non-root relation is not determined by the key of "
                                "that relation's view toward the root";
        if (o.planner == LMFAO_PLAN_FORCED)
          return fail(ctx, LMFAO_ERR_UNSUPPORTED, msg + " (root " + ctx->rels[bad_root].name + ")");
        std::vector<int> order((size_t)ctx->rels.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return ctx->rels[a].nrows > ctx->rels[b].nrows; });
        bool ok = false;
        for (int r : order) {
          if (r == bad_root) continue;
          lmfao_plan_opts o2 = o;
          o2.planner = LMFAO_PLAN_FORCED;
          o2.root_rel = r;
          o2.segment_rel = -2;
          build_plan(ctx, o2, false, nullptr);
          if (!views_carry_codes(*ctx->plan) || !(view_flags(ctx) & 1)) {
            ok = true;
            break;
          }
          drop_plan(ctx);
        }
        if (!ok) {
          // Per-query roots (Section 2: each query has its own root): every query takes the
          // largest relation whose views determine its group-by attributes, and the queries that
          // share a root form one physical plan; lmfao_run runs them all.
          const std::vector<QueryIn> all = ctx->queries;
          std::vector<int32_t> qroot(all.size(), -1);
          for (size_t q = 0; q < all.size(); ++q) {
            ctx->queries = {all[q]};
            for (int r : order) {
              lmfao_plan_opts o2 = o;
              o2.planner = LMFAO_PLAN_FORCED;
              o2.root_rel = r;
              o2.segment_rel = -2;
              build_plan(ctx, o2, false, nullptr);
              const bool good = !views_carry_codes(*ctx->plan) || !(view_flags(ctx) & 1);
              drop_plan(ctx);
              if (good) {
                qroot[q] = r;
                break;
              }
            }
            if (qroot[q] < 0) {
              ctx->queries = all;
              return fail(ctx, LMFAO_ERR_UNSUPPORTED, msg + " for any root relation (query " + std::to_string(q) + ")");
            }
          }
          std::map<int, std::vector<int>> by_root;
          for (size_t q = 0; q < all.size(); ++q) by_root[qroot[q]].push_back((int)q);
          std::vector<lmfao_subplan> subs;
          std::vector<std::pair<int, int>> route(all.size());
          for (auto &kv : by_root) {
            ctx->queries.clear();
            for (int q : kv.second) {
              route[q] = {(int)subs.size(), (int)ctx->queries.size()};
              ctx->queries.push_back(all[q]);
            }
            lmfao_plan_opts o2 = o;
            o2.planner = LMFAO_PLAN_FORCED;
            o2.root_rel = kv.first;
            o2.segment_rel = -2;
            try {
              build_plan(ctx, o2, false, nullptr);
            } catch (...) {
              for (auto &sp : subs) { sp.plan->arena.release(); delete sp.plan; }
              ctx->queries = all;
              throw;
            }
            subs.push_back(lmfao_subplan{ctx->plan, ctx->tree, kv.second});
            ctx->plan = nullptr;
          }
          ctx->queries = all;
          // the logical plan of the whole batch: one join tree, the per-query roots
          ctx->tree = build_tree(ctx, parent_links(ctx, o), largest_relation(ctx));
          ctx->logical = build_logical(ctx, ctx->tree, qroot.data());
          ctx->subs = std::move(subs);
          ctx->qroute = std::move(route);
          ctx->planned = true;
        }
      }
    }
    PhysPlan *P = ctx->plan ? ctx->plan : (ctx->subs.empty() ? nullptr : ctx->subs[0].plan);
    if (P && o.autotune && ctx->device >= 0 && ctx->plan) autotune(ctx, *P);
    if (P) P->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
      std::memset(info, 0, sizeof(*info));
      info->root_rel = ctx->tree.root;
      info->segment_rel = P ? P->segrel : -1;
      info->n_segments = P ? P->nseg : 0;
      info->n_views = (int)ctx->logical.views.size();
      info->n_groups = (int)ctx->logical.groups.size();
      int combine_kernels = P && !P->comb.empty() ? (P->use_c5 ? 2 : 1) : 0;
      if (P && !P->comb.empty() && !P->use_c3 && P->use_c4) {  // projection combine: several kernels
        const DComb4 &c4 = P->c4;
        combine_kernels = 1 + ((c4.need_d1 || c4.nent3) ? 1 : 0) + (c4.nent3 ? 1 : 0) + (c4.nent012 ? 1 : 0);
        for (int c = 1; c <= 3; ++c) combine_kernels += (c4.tab[c].nt + c4.tab[c].ng) ? 1 : 0;
      }
      info->n_kernels = P ? (int)P->vk.size() * 2 + 2 + combine_kernels + (P->fast.on ? 2 : 0) : 0;
      for (size_t i = 1; i < ctx->subs.size(); ++i) {  // the other plans of a batch with several roots
        const PhysPlan *Q = ctx->subs[i].plan;
        info->n_kernels += (int)Q->vk.size() * 2 + 2 + (Q->comb.empty() ? 0 : (Q->use_c5 ? 2 : 1)) + (Q->fast.on ? 2 : 0);
      }
      info->n_roots = ctx->subs.empty() ? 1 : (int)ctx->subs.size();
      info->mode = P ? P->mode : 0;
      info->predicted_ms = predicted;
      info->plan_ms = P ? P->plan_ms : 0;
      info->reorg_ms = P ? P->reorg_ms : 0;
      info->reorg_reused = P && P->reorg_cached ? 1 : 0;
    }
    return LMFAO_OK;
  });
}

int lmfao_plan_candidates(lmfao_ctx *ctx, const lmfao_plan_opts *opts, int32_t *cand, float *feats, int cap, int *n,
                          int *nfeat) {
  return guarded(ctx, [&]() -> int {
    if (ctx->device < 0) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "host-only context");
    if (ctx->rels.empty()) return fail(ctx, LMFAO_ERR_ARG, "no relations loaded");
    drop_plan(ctx);
    lmfao_plan_opts o = default_opts();
    if (opts) o = *opts;
    std::vector<Cand> cands = candidates(ctx, o);
    if (n) *n = (int)cands.size();
    if (nfeat) *nfeat = NFEAT;
    for (int c = 0; c < (int)cands.size() && c < cap; ++c) {
      if (cand) {
        cand[c * 4 + 0] = cands[c].root;
        cand[c * 4 + 1] = cands[c].seg;
        cand[c * 4 + 2] = cands[c].mode;
        cand[c * 4 + 3] = cands[c].combine;
      }
      if (feats) {
        std::vector<float> f;
        build_plan(ctx, cand_opts(o, cands[c]), true, &f);
        drop_plan(ctx);
        for (int k = 0; k < NFEAT; ++k) feats[(size_t)c * NFEAT + k] = f[k];
      }
    }
    return LMFAO_OK;
  });
}

int lmfao_run(lmfao_ctx *ctx, void *stream) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->planned || (!ctx->plan && ctx->subs.empty()))
      return fail(ctx, LMFAO_ERR_NOT_PLANNED, "lmfao_run before lmfao_plan (or on a host-only context)");
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->plan) enqueue_run(ctx, *ctx->plan, ctx->tree, s);
    for (auto &sp : ctx->subs) enqueue_run(ctx, *sp.plan, sp.tree, s);
    ctx->run_stream = s;
    ctx->ran = true;
    return LMFAO_OK;
  });
}

static void check_device_flags(lmfao_ctx *ctx) {
  int e = 0;
  LMFAO_CUDA(cudaStreamSynchronize(ctx->run_stream));
  std::vector<PhysPlan *> plans;
  if (ctx->plan) plans.push_back(ctx->plan);
  for (auto &sp : ctx->subs) plans.push_back(sp.plan);
  for (PhysPlan *P : plans) {
    int ep = 0;
    LMFAO_CUDA(cudaMemcpy(&ep, P->err, 4, cudaMemcpyDeviceToHost));
    e |= ep;
  }
  if (e & 1)
    throw Error(LMFAO_ERR_UNSUPPORTED,
                "a group-by attribute of a non-root relation is not determined by that relation's join key");
  if (e & 2) throw Error(LMFAO_ERR_UNSUPPORTED, "an exact count in a view exceeds 2^32");
  if (e & 8) throw Error(LMFAO_ERR_TIMEOUT, "a bounded wait of the block combine ran out (results incomplete)");
}

int lmfao_fetch(lmfao_ctx *ctx, int query_id, lmfao_result *out) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->ran || (!ctx->plan && ctx->subs.empty())) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "lmfao_fetch before lmfao_run");
    if (query_id < 0 || query_id >= (int)ctx->queries.size() || !out) return fail(ctx, LMFAO_ERR_ARG, "bad query id");
    check_device_flags(ctx);
    const auto pq = plan_of(ctx, query_id);
    PhysPlan &P = *pq.first;
    const QueryOut &q = P.qout[pq.second];
    std::vector<unsigned long long> ic(q.cells * (1 + q.naggs));
    std::vector<double> fs(q.cells * q.naggs);
    LMFAO_CUDA(cudaMemcpy(ic.data(), P.icnt + q.io, ic.size() * 8, cudaMemcpyDeviceToHost));
    if (!fs.empty()) LMFAO_CUDA(cudaMemcpy(fs.data(), P.fsum + q.fo, fs.size() * 8, cudaMemcpyDeviceToHost));
    int ng = (int)q.dom.size();
    ctx->fk.clear();
    ctx->fc.clear();
    ctx->fs.clear();
    int64_t groups = 0;
    for (int64_t c = 0; c < q.cells; ++c) {
      unsigned long long cnt = ic[c * (1 + q.naggs)];
      if (ng > 0 && cnt == 0) continue;
      ++groups;
      int64_t rem = c;
      std::vector<int32_t> key(ng);
      for (int i = ng - 1; i >= 0; --i) { key[i] = (int32_t)(rem % q.dom[i]); rem /= q.dom[i]; }
      ctx->fk.insert(ctx->fk.end(), key.begin(), key.end());
      ctx->fc.push_back((int64_t)cnt);
      for (int a = 0; a < q.naggs; ++a)
        ctx->fs.push_back(q.integral[a] ? (double)ic[c * (1 + q.naggs) + 1 + a] : fs[c * q.naggs + a]);
    }
    out->ngroups = groups;
    out->ngroupby = ng;
    out->naggs = q.naggs;
    out->group_keys = ctx->fk.data();
    out->counts = ctx->fc.data();
    out->sums = ctx->fs.data();
    return LMFAO_OK;
  });
}

int lmfao_result_device(lmfao_ctx *ctx, int query_id, int64_t *counts, double *sums, int64_t *ncells, void *stream) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->planned || (!ctx->plan && ctx->subs.empty())) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "no plan");
    if (query_id < 0 || query_id >= (int)ctx->queries.size()) return fail(ctx, LMFAO_ERR_ARG, "bad query id");
    const auto pq = plan_of(ctx, query_id);
    PhysPlan &P = *pq.first;
    const QueryOut &q = P.qout[pq.second];
    if (ncells) *ncells = q.cells;
    if (!counts && !sums) return LMFAO_OK;
    if (!ctx->ran) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "no run yet");
    cudaStream_t s = (cudaStream_t)stream;
    // integral flags of the query, uploaded once per plan (kept by the plan)
    int *fl;
    auto it = P.result_flags.find(pq.second);
    if (it == P.result_flags.end()) {
      fl = P.arena.upload(q.integral.empty() ? std::vector<int>{0} : q.integral, ctx->stream);
      LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
      P.result_flags[pq.second] = fl;
    } else fl = it->second;
    launch_results(P.icnt + q.io, P.fsum + q.fo, q.cells, q.naggs, fl, counts, sums, s);
    LMFAO_CUDA(cudaGetLastError());
    return LMFAO_OK;
  });
}

int lmfao_result_state(lmfao_ctx *ctx, int64_t **counts, int64_t *ncounts, double **sums, int64_t *nsums) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->subs.empty())
      return fail(ctx, LMFAO_ERR_UNSUPPORTED, "the batch is planned with several roots: one result state per plan");
    if (!ctx->planned || !ctx->plan) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "no plan");
    PhysPlan &P = *ctx->plan;
    if (counts) *counts = reinterpret_cast<int64_t *>(P.icnt);
    if (ncounts) *ncounts = P.nicnt;
    if (sums) *sums = P.fsum;
    if (nsums) *nsums = P.nfsum;
    return LMFAO_OK;
  });
}

int lmfao_describe_plan(lmfao_ctx *ctx, char *buf, size_t len, size_t *needed) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->planned) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "no plan");
    std::ostringstream o;
    const JoinTree &t = ctx->tree;
    const LogicalPlan &L = ctx->logical;
    auto nm = [&](int r) { return "\"" + json_escape(ctx->rels[r].name) + "\""; };
    o << "{\"relations\":[";
    for (size_t r = 0; r < ctx->rels.size(); ++r) o << (r ? "," : "") << nm((int)r);
    o << "],\"join_tree\":{\"root\":" << nm(t.root) << ",\"parent\":{";
    bool first = true;
    for (size_t r = 0; r < ctx->rels.size(); ++r) {
      if (t.parent[r] < 0) continue;
      o << (first ? "" : ",") << nm((int)r) << ":" << nm(t.parent[r]);
      first = false;
    }
    o << "}},\"query_roots\":[";
    for (size_t q = 0; q < L.query_root.size(); ++q) o << (q ? "," : "") << nm(L.query_root[q]);
    o << "],\"views\":[";
    for (size_t v = 0; v < L.views.size(); ++v) {
      const LogicalView &lv = L.views[v];
      o << (v ? "," : "") << "{\"from\":" << nm(lv.from) << ",\"to\":" << nm(lv.to) << ",\"key\":[";
      for (size_t i = 0; i < lv.key.size(); ++i) o << (i ? "," : "") << "\"" << json_escape(lv.key[i]) << "\"";
      o << "],\"aggregates\":[";
      size_t i = 0;
      for (auto &a : lv.aggs) o << (i++ ? "," : "") << "\"" << json_escape(a) << "\"";
      o << "],\"queries\":[";
      i = 0;
      for (int q : lv.queries) o << (i++ ? "," : "") << q;
      o << "],\"deps\":[";
      i = 0;
      for (int d : lv.deps) o << (i++ ? "," : "") << d;
      o << "]}";
    }
    o << "],\"groups\":[";
    for (size_t g = 0; g < L.groups.size(); ++g) {
      const LogicalGroup &lg = L.groups[g];
      o << (g ? "," : "") << "{\"node\":" << nm(lg.node) << ",\"views\":[";
      for (size_t i = 0; i < lg.views.size(); ++i) o << (i ? "," : "") << lg.views[i];
      o << "],\"queries\":[";
      for (size_t i = 0; i < lg.queries.size(); ++i) o << (i ? "," : "") << lg.queries[i];
      o << "],\"deps\":[";
      size_t i = 0;
      for (int d : lg.deps) o << (i++ ? "," : "") << d;
      o << "]}";
    }
    const PhysPlan *PP = ctx->plan ? ctx->plan : (ctx->subs.empty() ? nullptr : ctx->subs[0].plan);
    o << "],\"physical_roots\":[";
    if (ctx->plan) o << "{\"root\":" << nm(ctx->plan->root) << ",\"queries\":\"all\"}";
    for (size_t i = 0; i < ctx->subs.size(); ++i) {
      o << (i ? "," : "") << "{\"root\":" << nm(ctx->subs[i].plan->root) << ",\"queries\":[";
      for (size_t k = 0; k < ctx->subs[i].qids.size(); ++k) o << (k ? "," : "") << ctx->subs[i].qids[k];
      o << "]}";
    }
    if (!PP) {
      o << "],\"physical\":null}";
      std::string str = o.str();
      if (needed) *needed = str.size() + 1;
      if (buf && len) {
        size_t m = std::min(len - 1, str.size());
        std::memcpy(buf, str.data(), m);
        buf[m] = 0;
      }
      return LMFAO_OK;
    }
    const PhysPlan &P = *PP;
    o << "],\"physical\":{\"root\":" << nm(P.root) << ",\"segment_relation\":"
      << (P.segrel >= 0 ? nm(P.segrel) : std::string("null")) << ",\"n_segments\":" << P.nseg
      << ",\"outer\":[";
    for (size_t i = 0; i < P.outer.size(); ++i) o << (i ? "," : "") << nm(P.outer[i]);
    o << "],\"inner\":[";
    for (size_t i = 0; i < P.inner.size(); ++i) o << (i ? "," : "") << nm(P.inner[i]);
    o << "],\"precision\":\"" << (P.fp64 ? "fp64" : P.split_bf16 ? "split_bf16" : "fp32") << "\",\"mode\":\""
      << (P.mode == LMFAO_MODE_PER_TUPLE ? "per_tuple" : P.fast.on ? "factorised" : "generic")
      << "\",\"specialised_pass\":" << (P.fast.on ? "true" : "false") << ",\"specialised_pass_declined\":\""
      << json_escape(P.fast.on ? "" : P.fast_why) << "\""
      << ",\"lean_pass\":" << (P.fast.on && P.fast.lean ? "true" : "false")
      << ",\"block_combine\":" << (P.use_c3 ? "true" : "false") << ",\"prefix_digits\":" << P.prefix_len
      << ",\"block_combine_two_kernels\":" << (P.use_c5 ? "true" : "false") << ",\"contraction\":\""
      << (!P.use_c5 ? (P.use_c3 ? "cuda cores, single kernel" : "none")
                    : P.c5.tc ? "tensor cores (tcgen05, split BF16)"
                              : std::string(P.fp64 ? "cuda cores FP64" : "cuda cores FP32") +
                                    (P.c5.pipe ? ", dense B operand, cp.async pipeline"
                                               : P.c5.dense ? ", dense B operand" : ""))
      << "\",\"combine_chunk\":" << P.c5.kc << ",\"combine_bulk_copies\":" << (P.c5.bulk ? "true" : "false")
      << ",\"combine_blocks\":" << P.c3.nblocks << ",\"combine_entries\":" << P.c3.nent
      << ",\"block_terms\":[" << P.c3.na << "," << P.c3.nb << "," << P.c3.nbi << "]"
      << ",\"y_columns\":[" << P.c3.nyf << "," << P.c3.nyi << "]"
      << ",\"combine_note\":\"" << json_escape(P.c5_why) << "\""
      << ",\"combine_z_bytes\":" << combine_z_bytes(P) << ",\"combine_z_flops\":" << combine_z_flops(P)
      << ",\"projection_combine\":" << (!P.use_c3 && P.use_c4 ? "true" : "false")
      << ",\"projection_entries\":[" << P.c4.nent012 << "," << P.c4.nent3 << "," << P.c4.njobs << "]"
      << ",\"projection_stream\":" << (P.use_c4 && P.c4.stream ? "true" : "false")
      << ",\"projection_stream_tile\":[" << P.c4.c1 << "," << P.c4.c0 << "," << P.c4.nx << "," << P.c4.ny << "]"
      << ",\"projection_fused_class3\":" << (P.use_c4 && P.c4.stream && P.c4.fused3 ? "true" : "false")
      << ",\"filter_family\":" << P.fast.fam_k << ",\"cta_items\":" << P.fast.b4.size()
      << ",\"segment_sums\":" << P.b0f.size() + P.b0i.size()
      << ",\"combine_items\":" << P.comb.size() << ",\"per_tuple_items\":" << P.b2.size()
      << ",\"outer_terms\":" << P.psis.size() << ",\"row_terms\":" << P.rts.size() << ",\"work_items\":" << P.nwork
      << ",\"fact_pass_bytes\":" << fact_pass_bytes(ctx, P) << ",\"root_rows\":" << ctx->rels[P.root].nrows
      << ",\"tiles\":{\"work_chunk\":" << P.work_chunk << ",\"combine_chunk\":" << (P.use_c5 ? P.c5.kc : 0)
      << ",\"root_pass_lanes\":" << (P.fd.lanes ? "\"tuple per lane\"" : "\"quad per lane\"")
      << ",\"root_pass_grid\":" << P.fast_grid << ",\"root_pass_block\":" << (P.gen.fn ? P.gen.block : P.fast_block)
      << ",\"autotuned\":" << (P.tuned ? "true" : "false") << ",\"from_cache\":" << (P.tune_cached ? "true" : "false")
      << ",\"candidates\":" << P.tune_candidates << ",\"tune_ms\":" << P.tune_ms << "}"
      << ",\"reorganisation_ms\":" << P.reorg_ms << ",\"reorganisation_reused\":" << (P.reorg_cached ? "true" : "false");
    if (P.fast.on) {
      const DFast &d = P.fd;
      o << ",\"root_pass\":{\"monomials\":" << d.nm << ",\"inner_columns\":" << d.nw << ",\"value_columns\":" << d.nx
        << ",\"inner_keys\":" << d.nkeys << ",\"inner_codes\":" << d.ncode << ",\"histograms\":" << d.nb1
        << ",\"hist_cells_per_warp\":" << d.hist_i + d.hist_f << ",\"root_to_inner_columns\":" << d.n3
        << ",\"root_to_inner_float\":" << d.n3f << ",\"root_to_inner_integral\":" << d.n3i
        << ",\"shared_partials\":" << d.smem_p << ",\"shared_view\":" << d.smem_view
        << ",\"smem_bytes\":" << fast_smem(d, P.fp64, P.fast_block) << ",\"block\":" << P.fast_block
        << ",\"grid\":" << P.fast_grid << ",\"vector_loads\":" << d.vec
        << ",\"generated\":" << (P.gen.fn ? "true" : "false") << ",\"generated_block\":" << P.gen.block
        << ",\"generated_smem\":" << P.gen.smem << ",\"source_hash\":\"" << (P.gen.fn ? P.gen.source_hash : "")
        << "\",\"not_generated_because\":\"" << json_escape(P.gen.why)
        << "\"}";
    }
    o
      << ",\"view_columns\":{";
    first = true;
    for (int r : t.post) {
      o << (first ? "" : ",") << nm(r) << ":" << P.views[r].cols.size();
      first = false;
    }
    o << "}}}";
    std::string str = o.str();
    if (needed) *needed = str.size() + 1;
    if (buf && len) {
      size_t m = std::min(len - 1, str.size());
      std::memcpy(buf, str.data(), m);
      buf[m] = 0;
    }
    return LMFAO_OK;
  });
}

int lmfao_cart_variances(lmfao_ctx *ctx, const int *qids, int n, double *out, void *stream) {
  return guarded(ctx, [&]() -> int {
    if (n < 0 || (n && (!qids || !out))) return fail(ctx, LMFAO_ERR_ARG, "bad arguments");
    std::vector<int64_t> qd((size_t)std::max(n, 0) * kCartDescWords);
    PhysPlan *PP = nullptr;
    const int nb = cart_descriptors(ctx, qids, n, qd.data(), &PP);
    if (!n || nb < 2) return LMFAO_OK;
    PhysPlan &P = *PP;
    check_device_flags(ctx);  // the run's own failures (counts above 2^32, a wait that ran out)
    int64_t *dq = P.arena.upload(qd, ctx->stream);
    LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
    launch_cart_variances(P.icnt, P.fsum, dq, n, nb, out, (cudaStream_t)stream);
    LMFAO_CUDA(cudaGetLastError());
    return LMFAO_OK;
  });
}

int lmfao_cart_tree(lmfao_ctx *ctx, const char *target, const char *const *features, int nfeatures,
                    const float *thresholds, const int32_t *nthresholds, int depth, const lmfao_plan_opts *opts,
                    lmfao_cart_node *nodes, double *level_ms) {
  return guarded(ctx, [&]() -> int {
    if (ctx->device < 0) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "host-only context");
    if (!target || !features || nfeatures <= 0 || !thresholds || !nthresholds || !nodes || depth < 1 || depth > 5)
      return fail(ctx, LMFAO_ERR_ARG, "bad tree arguments");
    std::vector<std::vector<float>> thr(nfeatures);
    int64_t off = 0;
    for (int f = 0; f < nfeatures; ++f) {
      if (!features[f] || nthresholds[f] < 1 || nthresholds[f] > 31) return fail(ctx, LMFAO_ERR_ARG, "bad feature thresholds");
      thr[f].assign(thresholds + off, thresholds + off + nthresholds[f]);
      off += nthresholds[f];
      for (size_t k = 1; k < thr[f].size(); ++k)
        if (!(thr[f][k - 1] < thr[f][k])) return fail(ctx, LMFAO_ERR_ARG, "thresholds must be strictly ascending");
    }
    const int nnodes_all = (1 << depth) - 1;
    for (int i = 0; i < nnodes_all; ++i) nodes[i] = lmfao_cart_node{0, -1, 0.f, 0.0, 0, 0.0, 0.0};
    std::vector<std::vector<PredIn>> path(nnodes_all);
    nodes[0].active = 1;
    for (int lev = 0; lev < depth; ++lev) {
      const auto t0 = std::chrono::steady_clock::now();
      std::vector<int> act;
      for (int v = (1 << lev) - 1; v < (1 << (lev + 1)) - 1; ++v)
        if (nodes[v].active) act.push_back(v);
      if (act.empty()) {
        if (level_ms) level_ms[2 * lev] = level_ms[2 * lev + 1] = 0;
        continue;
      }
      drop_plan(ctx);
      ctx->queries.clear();
      for (int v : act)
        for (int f = 0; f < nfeatures; ++f) {
          QueryIn q;
          q.aggs = {{}, {FactorIn{target, LMFAO_FN_ID, 1}}, {FactorIn{target, LMFAO_FN_POW, 2}}};
          q.gb = {GroupIn{features[f], LMFAO_GB_BUCKET, thr[f]}};
          q.filters = path[v];
          ctx->queries.push_back(q);
        }
      int rc = lmfao_plan(ctx, opts, nullptr);
      if (rc != LMFAO_OK) return rc;
      if (!ctx->plan) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "a tree level needs several roots");
      const auto t1 = std::chrono::steady_clock::now();
      PhysPlan &P = *ctx->plan;
      enqueue_run(ctx, P, ctx->tree, ctx->stream);
      ctx->run_stream = ctx->stream;
      ctx->ran = true;
      const int nq = (int)ctx->queries.size();
      std::vector<int> ids(nq);
      std::iota(ids.begin(), ids.end(), 0);
      std::vector<int64_t> qd((size_t)nq * kCartDescWords);
      for (int i = 0; i < nq; ++i) {
        const QueryOut &qo = P.qout[i];
        int64_t *d = qd.data() + (size_t)i * kCartDescWords;
        d[0] = qo.io;
        d[1] = qo.fo;
        d[2] = qo.cells;
        d[3] = qo.naggs;
        d[4] = 1;
        d[5] = 2;
      }
      std::vector<int> qbeg(act.size() + 1);
      for (size_t i = 0; i <= act.size(); ++i) qbeg[i] = (int)i * nfeatures;
      int64_t *dq = P.arena.upload(qd, ctx->stream);
      int *dqb = P.arena.upload(qbeg, ctx->stream);
      int2 *dbest = (int2 *)P.arena.alloc(act.size() * sizeof(int2));
      double *dscore = (double *)P.arena.alloc(act.size() * 8);
      double *dstats = (double *)P.arena.alloc(act.size() * 3 * 8);
      launch_cart_split(P.icnt, P.fsum, dq, dqb, (int)act.size(), dbest, dscore, dstats, ctx->stream);
      LMFAO_CUDA(cudaGetLastError());
      check_device_flags(ctx);
      std::vector<int2> best(act.size());
      std::vector<double> score(act.size()), stats(3 * act.size());
      LMFAO_CUDA(cudaMemcpy(best.data(), dbest, best.size() * sizeof(int2), cudaMemcpyDeviceToHost));
      LMFAO_CUDA(cudaMemcpy(score.data(), dscore, score.size() * 8, cudaMemcpyDeviceToHost));
      LMFAO_CUDA(cudaMemcpy(stats.data(), dstats, stats.size() * 8, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < act.size(); ++i) {
        const int v = act[i];
        lmfao_cart_node &nd = nodes[v];
        nd.count = (int64_t)stats[3 * i];
        nd.sum_y = stats[3 * i + 1];
        nd.sum_y2 = stats[3 * i + 2];
        if (best[i].x < 0) continue;
        nd.feature = best[i].x;
        nd.threshold = thr[nd.feature][best[i].y];
        nd.score = score[i];
        if (2 * v + 2 < nnodes_all) {
          for (int c = 0; c < 2; ++c) {
            path[2 * v + 1 + c] = path[v];
            path[2 * v + 1 + c].push_back(PredIn{features[nd.feature], c ? LMFAO_GT : LMFAO_LE, nd.threshold});
            nodes[2 * v + 1 + c].active = 1;
          }
        }
      }
      const auto t2 = std::chrono::steady_clock::now();
      if (level_ms) {
        level_ms[2 * lev] = std::chrono::duration<double, std::milli>(t1 - t0).count();
        level_ms[2 * lev + 1] = std::chrono::duration<double, std::milli>(t2 - t1).count();
      }
    }
    drop_plan(ctx);
    ctx->queries.clear();
    return LMFAO_OK;
  });
}

int lmfao_ridge_fit(lmfao_ctx *ctx, int query_id, const char *target, const char *const *features, int nfeatures,
                    double lambda, int method, int iters, double step, double *theta, double *loss,
                    double *grad_norm) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->ran || (!ctx->plan && ctx->subs.empty())) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "no run yet");
    if (query_id < 0 || query_id >= (int)ctx->queries.size() || !target || !theta || nfeatures < 0 ||
        (nfeatures && !features) || nfeatures > 126 || lambda < 0 || (method != LMFAO_RIDGE_CLOSED_FORM &&
        method != LMFAO_RIDGE_BGD) || (method == LMFAO_RIDGE_BGD && (iters < 0 || !(step > 0))))
      return fail(ctx, LMFAO_ERR_ARG, "bad ridge arguments");
    const QueryIn &Q = ctx->queries[query_id];
    if (!Q.gb.empty() || !Q.filters.empty())
      return fail(ctx, LMFAO_ERR_ARG, "the ridge query must be ungrouped and unfiltered");
    // canonical form of a product: attribute -> power
    auto key_of = [](const std::vector<FactorIn> &fs) {
      std::map<std::string, int> k;
      for (const FactorIn &f : fs) k[f.attr] += f.fn == LMFAO_FN_POW ? f.param : 1;
      return k;
    };
    std::map<std::map<std::string, int>, int> agg;
    for (int a = 0; a < (int)Q.aggs.size(); ++a) agg.emplace(key_of(Q.aggs[a]), a);
    std::vector<std::string> z{""};  // z_0 = 1 (the intercept)
    for (int f = 0; f < nfeatures; ++f) {
      if (!features[f]) return fail(ctx, LMFAO_ERR_ARG, "null feature name");
      z.push_back(features[f]);
    }
    z.push_back(target);
    const int d = nfeatures, w = d + 2;
    std::vector<int> zmap((size_t)w * w, -1);
    const auto pq = plan_of(ctx, query_id);
    const QueryOut &qo = pq.first->qout[pq.second];
    for (int i = 0; i < w; ++i)
      for (int j = 0; j < w; ++j) {
        if (i == 0 && j == 0) continue;  // the COUNT of the (single) group
        std::map<std::string, int> k;
        if (i) k[z[i]] += 1;
        if (j) k[z[j]] += 1;
        auto it = agg.find(k);
        if (it == agg.end() || qo.integral[it->second]) {
          std::string name;
          for (auto &kv : k) name += (name.empty() ? "" : " * ") + kv.first + (kv.second > 1 ? "^2" : "");
          return fail(ctx, LMFAO_ERR_ARG, "the ridge query has no SUM(" + name + ")");
        }
        zmap[(size_t)i * w + j] = it->second;
      }
    check_device_flags(ctx);
    PhysPlan &P = *pq.first;
    int *dz = P.arena.upload(zmap, ctx->stream);
    double *dout = (double *)P.arena.alloc((size_t)(d + 3) * 8);
    launch_ridge(P.icnt, P.fsum, qo.io, qo.fo, dz, d, lambda, method, iters, step, dout, ctx->stream);
    LMFAO_CUDA(cudaGetLastError());
    std::vector<double> out(d + 3);
    LMFAO_CUDA(cudaMemcpyAsync(out.data(), dout, out.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    LMFAO_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i <= d; ++i) theta[i] = out[i];
    if (loss) *loss = out[d + 1];
    if (grad_norm) *grad_norm = out[d + 2];
    return LMFAO_OK;
  });
}

int lmfao_group_count(lmfao_ctx *ctx, const lmfao_groupby *gb, int ngb, int64_t cap, int32_t *keys, int64_t *counts,
                      int64_t *ngroups) {
  return guarded(ctx, [&]() -> int {
    if (ctx->device < 0) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "host-only context");
    if (ctx->rels.empty()) return fail(ctx, LMFAO_ERR_ARG, "no relations loaded");
    if (!gb || ngb < 1 || ngb > GC_MAXATTR || cap < 0 || (cap > 0 && (!keys || !counts)) || !ngroups)
      return fail(ctx, LMFAO_ERR_ARG, "bad group-count arguments");
    cudaStream_t s = ctx->stream;
    lmfao_plan_opts o = default_opts();
    const std::vector<int> par = parent_links(ctx, o);
    const JoinTree t = build_tree(ctx, par, largest_relation(ctx));
    // group attributes: home relation, code kind and domain
    struct Attr { int rel, col, kind, nthr; int64_t dom, radix; float *thr; };
    std::vector<Attr> at(ngb);
    std::vector<void *> tmp;
    auto dalloc = [&](size_t bytes) {
      void *p = nullptr;
      LMFAO_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
      tmp.push_back(p);
      return p;
    };
    struct Free {  // temporaries of this call
      std::vector<void *> &v;
      ~Free() {
        for (void *p : v) cudaFree(p);
      }
    } free_tmp{tmp};
    for (int i = 0; i < ngb; ++i) {
      if (!gb[i].attr) return fail(ctx, LMFAO_ERR_ARG, "null group attribute");
      Attr &a = at[i];
      a.rel = home_of(ctx, t, gb[i].attr);
      a.col = ctx->rels[a.rel].col(gb[i].attr);
      const Column &c = ctx->rels[a.rel].cols[a.col];
      a.thr = nullptr;
      a.nthr = 0;
      if (gb[i].kind == LMFAO_GB_VALUE) {
        if (c.role != LMFAO_CONT) { a.kind = 0; a.dom = c.domain; }
        else if (c.dtype == LMFAO_U8) { a.kind = 0; a.dom = 256; }
        else { a.kind = 2; a.dom = int64_t(1) << 32; }  // the FP32 value itself (its bit pattern)
      } else if (gb[i].kind == LMFAO_GB_BUCKET) {
        if (gb[i].nthresholds < 0 || (gb[i].nthresholds && !gb[i].thresholds)) return fail(ctx, LMFAO_ERR_ARG, "bad thresholds");
        for (int k = 1; k < gb[i].nthresholds; ++k)
          if (!(gb[i].thresholds[k - 1] < gb[i].thresholds[k])) return fail(ctx, LMFAO_ERR_ARG, "thresholds must be strictly ascending");
        a.kind = 1;
        a.nthr = gb[i].nthresholds;
        a.dom = a.nthr + 1;
        a.thr = (float *)dalloc((size_t)a.nthr * 4);
        if (a.nthr) LMFAO_CUDA(cudaMemcpyAsync(a.thr, gb[i].thresholds, (size_t)a.nthr * 4, cudaMemcpyHostToDevice, s));
      } else return fail(ctx, LMFAO_ERR_ARG, "unknown group-by kind");
    }
    double total = 1;
    for (int i = ngb - 1; i >= 0; --i) {
      at[i].radix = (int64_t)total;
      total *= (double)at[i].dom;
    }
    if (total > 4.6e18) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "the group key does not fit 62 bits");
    auto fill_cols = [&](DGcRel &d, int r) {
      const Relation &R = ctx->rels[r];
      if ((int)R.cols.size() > GC_MAXCOL) throw Error(LMFAO_ERR_UNSUPPORTED, "relation with more than 32 columns");
      d.nrows = R.nrows;
      for (size_t c = 0; c < R.cols.size(); ++c) d.col[c] = dcol(R.cols[c]);
      d.nattr = 0;
      for (const Attr &a : at)
        if (a.rel == r) d.attr[d.nattr++] = DGcAttr{a.kind, a.col, a.nthr, a.thr, a.radix};
    };
    // the join key of relation r toward relation p: columns of `side` and mixed-radix strides
    auto join_key = [&](int r, int p, int side, int *kcol, int64_t *kstride) {
      const std::vector<std::string> sh = shared_attrs(ctx, r, p);
      if (sh.empty() || (int)sh.size() > MAXK) throw Error(LMFAO_ERR_UNSUPPORTED, "join key of 0 or more than 4 attributes");
      int64_t nk = 1;
      for (int i = (int)sh.size() - 1; i >= 0; --i) {
        const Column &c = ctx->rels[r].cols[ctx->rels[r].col(sh[i])];
        if (c.role == LMFAO_CONT) throw Error(LMFAO_ERR_UNSUPPORTED, "join on a value attribute");
        kcol[i] = ctx->rels[side].col(sh[i]);
        kstride[i] = nk;
        nk *= c.domain;
        if (nk > (int64_t(1) << 28)) throw Error(LMFAO_ERR_UNSUPPORTED, "join key domain above 2^28");
      }
      return std::make_pair((int)sh.size(), nk);
    };
    std::vector<unsigned long long *> vcnt(ctx->rels.size(), nullptr);
    std::vector<long long *> vcode(ctx->rels.size(), nullptr);
    int *err = (int *)dalloc(4);
    LMFAO_CUDA(cudaMemsetAsync(err, 0, 4, s));
    auto add_children = [&](DGcRel &d, int r) {
      d.nchild = 0;
      for (int c : t.children[r]) {
        if (d.nchild >= MAXCH) throw Error(LMFAO_ERR_UNSUPPORTED, "more than 8 children");
        DGcChild &ch = d.child[d.nchild++];
        ch.nk = join_key(c, r, r, ch.kcol, ch.kstride).first;
        ch.cnt = vcnt[c];
        ch.code = vcode[c];
      }
    };
    for (int r : t.post) {
      DGcRel d{};
      fill_cols(d, r);
      const auto k = join_key(r, t.parent[r], r, d.kcol, d.kstride);
      d.nk = k.first;
      add_children(d, r);
      vcnt[r] = (unsigned long long *)dalloc((size_t)k.second * 8);
      vcode[r] = (long long *)dalloc((size_t)k.second * 8);
      LMFAO_CUDA(cudaMemsetAsync(vcnt[r], 0, (size_t)k.second * 8, s));
      LMFAO_CUDA(cudaMemsetAsync(vcode[r], 0xff, (size_t)k.second * 8, s));
      d.cnt = vcnt[r];
      d.code = vcode[r];
      launch_gc_view(d, err, s);
    }
    // the global table: twice the largest possible number of groups, rounded up to 2^k
    const double most = std::min<double>(total, (double)std::max<int64_t>(1, ctx->rels[t.root].nrows));
    int64_t slots = 1024;
    while ((double)slots < 2 * most && slots < (int64_t(1) << 28)) slots *= 2;
    unsigned long long *gk = (unsigned long long *)dalloc((size_t)slots * 8);
    unsigned long long *gc = (unsigned long long *)dalloc((size_t)slots * 8);
    LMFAO_CUDA(cudaMemsetAsync(gk, 0xff, (size_t)slots * 8, s));
    LMFAO_CUDA(cudaMemsetAsync(gc, 0, (size_t)slots * 8, s));
    DGcRel d{};
    fill_cols(d, t.root);
    add_children(d, t.root);
    launch_gc_root(d, gk, gc, (unsigned long long)(slots - 1), err, s);
    DGcOut out{};
    out.ngb = ngb;
    for (int i = 0; i < ngb; ++i) out.radix[i] = at[i].radix;
    out.cap = cap;
    out.keys = keys;
    out.counts = counts;
    unsigned long long *nout = (unsigned long long *)dalloc(8);
    LMFAO_CUDA(cudaMemsetAsync(nout, 0, 8, s));
    launch_gc_compact(gk, gc, slots, out, nout, s);
    LMFAO_CUDA(cudaGetLastError());
    int e = 0;
    unsigned long long n = 0;
    LMFAO_CUDA(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s));
    LMFAO_CUDA(cudaMemcpyAsync(&n, nout, 8, cudaMemcpyDeviceToHost, s));
    LMFAO_CUDA(cudaStreamSynchronize(s));
    if (e & 1) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "a group attribute of a non-root relation is not determined by its join key");
    if (e & 4) return fail(ctx, LMFAO_ERR_UNSUPPORTED, "more groups than the hash table holds");
    *ngroups = (int64_t)n;
    return LMFAO_OK;
  });
}

int lmfao_set_profiling(lmfao_ctx *ctx, int on) {
  return guarded(ctx, [&]() -> int {
    ctx->profiling = on != 0;
    return LMFAO_OK;
  });
}

int lmfao_kernel_times(lmfao_ctx *ctx, double *ms, int cap, int *n) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->ran) return fail(ctx, LMFAO_ERR_NOT_PLANNED, "no run yet");
    LMFAO_CUDA(cudaStreamSynchronize(ctx->run_stream));
    int k = (int)ctx->ev_names.size() - 1;
    if (k < 0) k = 0;
    ctx->kernel_names.assign(ctx->ev_names.begin() + (ctx->ev_names.empty() ? 0 : 1), ctx->ev_names.end());
    for (int i = 0; i < k && i < cap; ++i) {
      float f = 0;
      LMFAO_CUDA(cudaEventElapsedTime(&f, ctx->events[i], ctx->events[i + 1]));
      ms[i] = f;
    }
    if (n) *n = k;
    return LMFAO_OK;
  });
}

const char *lmfao_kernel_name(lmfao_ctx *ctx, int i) {
  if (!ctx || i < 0 || i >= (int)ctx->kernel_names.size()) return "";
  return ctx->kernel_names[i].c_str();
}

}  // extern "C"
