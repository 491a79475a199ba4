// Plan-specialised lean root pass, generated as CUDA source and compiled with NVRTC.
//
// The generated kernel computes exactly what lean_pass_kernel computes for the same DFast
// (per-segment sums of basis monomials x inner view columns, per-segment inner-code
// histograms, root-to-inner partials), with the shape of the batch folded in:
//   * the inner view rows are staged in shared memory with the histogram codes of the row
//     packed behind its values (FP32: as int bits in the same 16-byte vectors), as planes of
//     16-byte parts, so one tuple reads its row with ceil(row/4) vector loads that spread over
//     all shared-memory banks;
//   * per tuple the code is straight-line: the basis monomials, one multiply-add per
//     (monomial, view column), one shared atomic per histogram set and per root-to-inner
//     column, with every index a constant;
//   * a work item's full 4-tuple quads are read with 16-byte loads and no range checks; the
//     at most 6 tuples of its ragged head and tail are taken by single lanes;
//   * each CTA takes a contiguous range of work items with about 1/G of the tuples (tuple
//     quantiles of the work list) and hands them to its warps with a ticket in shared memory
//     (one global counter for all warps of the GPU was a serial point);
//   * the next item's ticket and record are requested when the current item starts, and its
//     weight and first quad while the segment sums of the current one are reduced.
#include "codegen.h"

#include <nvrtc.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <sstream>

namespace lmfao {

namespace {

enum Arg {
  A_NWORK, A_WORK, A_WSEG, A_WORKQ, A_TABLE, A_CODES, A_PHI0F, A_PHI0I, A_PHI1I, A_P3F, A_P3I, A_KC, A_X0,
  A_NARGS = A_X0 + 3
};

struct GenArgs {
  unsigned long long v[16];
};
static_assert(A_NARGS <= 16, "argument slots");

int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct Shape {
  bool fp64;
  int block, nx, ni, nw, nm, nb1, ncode, n3, n3f, n3i, n0i, hist, rs;
  int nfull, tew;  // FP32 rows: full 16-byte planes and the element width (words) of the tail plane
  long long nkeys, phi1i_seg;
  int xdt[3];
  size_t off_tab, off_code, off_pf, off_pi, off_h, smem;
};

Shape shape_of(const DFast &d, bool fp64, int block) {
  Shape s{};
  s.fp64 = fp64;
  s.block = block;
  s.nx = d.nx;
  s.ni = d.ni;
  s.nw = d.ni ? d.nw : 1;
  s.nm = 1 + d.nx + d.nx * (d.nx + 1) / 2;
  s.nb1 = d.nb1;
  s.ncode = d.ncode;
  s.n3 = d.n3;
  s.n3f = d.n3f;
  s.n3i = d.n3i;
  s.n0i = d.n0i;
  s.hist = d.hist_i;
  s.nkeys = d.ni ? d.nkeys : 0;
  s.phi1i_seg = d.phi1i_seg;
  for (int i = 0; i < 3; ++i) s.xdt[i] = i < d.nx ? d.col[d.xslot[i]].dtype : LMFAO_F32;
  const size_t ts = fp64 ? 8 : 4;
  s.rs = fp64 ? round_up(s.nw, 2) : round_up(s.nw + s.nb1, 4);
  {
    const int rw = s.nw + s.nb1, tw = rw % 4;
    s.nfull = rw / 4;
    s.tew = tw == 3 ? 4 : tw;  // a row tail of 1 or 2 words is read with a 4- or 8-byte load
  }
  size_t off = 0;
  auto region = [&](size_t bytes) {
    size_t at = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return at;
  };
  s.off_tab = region(fp64 ? ts * (size_t)s.nkeys * s.rs : 4 * (size_t)s.nkeys * (4 * s.nfull + s.tew));
  s.off_code = region(fp64 ? 4 * (size_t)s.nkeys * s.nb1 : 0);
  s.off_pf = region(ts * (size_t)s.nkeys * s.n3f);
  s.off_pi = region(4 * (size_t)s.nkeys * s.n3i);
  s.off_h = region(4 * (size_t)(block / 32) * s.hist);
  s.smem = off;
  return s;
}

// The monomial u_j of the degree <= 2 basis over x0..x{nx-1}: 1, x_i, x_i x_j (i <= j).
std::string basis_expr(int nx, int j) {
  if (j == 0) return "(T)1";
  if (j <= nx) return "x" + std::to_string(j - 1);
  int q = 1 + nx;
  for (int a = 0; a < nx; ++a)
    for (int b = a; b < nx; ++b, ++q)
      if (q == j) return "x" + std::to_string(a) + " * x" + std::to_string(b);
  return "(T)0";
}

// one component of a 4-tuple register of a value column
std::string x_component(int dt, const std::string &reg, int i) {
  static const char *c[4] = {"x", "y", "z", "w"};
  if (dt == LMFAO_U8) return "(T)((" + reg + " >> " + std::to_string(8 * i) + ") & 0xffu)";
  return "(T)" + reg + "." + c[i];
}

}  // namespace

WarpReduce gen_warp_reduce(int V, const std::string &ind) {
  WarpReduce w{};
  w.V = V;
  std::ostringstream o;
  if (V <= 32) {
    int L = 0;
    while ((1 << L) < V) ++L;
    const int PV = 1 << L;
    w.F = 1;
    w.shift = 5 - L;
    o << ind << "T r_[" << PV << "];\n";
    o << "#pragma unroll\n" << ind << "for (int i = 0; i < " << PV << "; ++i) r_[i] = i < " << V << " ? acc[i < " << V
      << " ? i : 0] : (T)0;\n";
    if (L > 0) {
      o << "#pragma unroll\n" << ind << "for (int lvl = 0; lvl < " << L << "; ++lvl) {\n";
      o << ind << "  const int o = 16 >> lvl, h = " << PV << " >> (lvl + 1);\n";
      o << ind << "  const bool up = (lane & o) != 0;\n";
      o << "#pragma unroll\n" << ind << "  for (int i = 0; i < h; ++i) {\n";
      o << ind << "    const T send = up ? r_[i] : r_[i + h];\n";
      o << ind << "    const T keep = up ? r_[i + h] : r_[i];\n";
      o << ind << "    r_[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);\n" << ind << "  }\n" << ind << "}\n";
    }
    for (int b = (16 >> L); b >= 1; b >>= 1) o << ind << "r_[0] += __shfl_xor_sync(0xffffffffu, r_[0], " << b << ");\n";
  } else {
    w.F = (V + 31) / 32;
    w.shift = 0;
    const int PV = 32 * w.F;
    o << ind << "T r_[" << PV << "];\n";
    o << "#pragma unroll\n" << ind << "for (int i = 0; i < " << PV << "; ++i) r_[i] = i < " << V << " ? acc[i < " << V
      << " ? i : 0] : (T)0;\n";
    o << "#pragma unroll\n" << ind << "for (int lvl = 0; lvl < 5; ++lvl) {\n";
    o << ind << "  const int o = 16 >> lvl, h = " << PV << " >> (lvl + 1);\n";
    o << ind << "  const bool up = (lane & o) != 0;\n";
    o << "#pragma unroll\n" << ind << "  for (int i = 0; i < h; ++i) {\n";
    o << ind << "    const T send = up ? r_[i] : r_[i + h];\n";
    o << ind << "    const T keep = up ? r_[i + h] : r_[i];\n";
    o << ind << "    r_[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);\n" << ind << "  }\n" << ind << "}\n";
  }
  w.src = o.str();
  return w;
}

std::string gen_reduce_flush(const WarpReduce &w, const std::string &dst, const std::string &base,
                             const std::string &ind) {
  std::ostringstream o;
  if (w.F == 1) {
    const int mask = (1 << w.shift) - 1;
    o << ind << "{ const int i = lane >> " << w.shift << "; if (" << (mask ? "(lane & " + std::to_string(mask) + ") == 0 && " : "")
      << "i < " << w.V << " && r_[0] != (T)0) atomicAdd(" << dst << " + " << base << " + i, r_[0]); }\n";
  } else {
    for (int e = 0; e < w.F; ++e)
      o << ind << "{ const int i = lane * " << w.F << " + " << e << "; if (i < " << w.V << " && r_[" << e
        << "] != (T)0) atomicAdd(" << dst << " + " << base << " + i, r_[" << e << "]); }\n";
  }
  return o.str();
}

std::string gen_root_pass_source(const DFast &d, bool fp64, int block) {
  const Shape s = shape_of(d, fp64, block);
  const int V = s.nm * s.nw;
  std::ostringstream o;
  o << "// generated lean root pass\n";
  o << "typedef " << (fp64 ? "double" : "float") << " T;\n";
  o << "struct GenArgs { unsigned long long v[16]; };\n";
  o << "struct Work { long long r0; int seg; int len; };\n";
  // per-tuple body
  o << "__device__ __forceinline__ void tuple(const int k";
  for (int i = 0; i < 3; ++i) o << ", const T x" << i;
  o << ", T (&acc)[" << V << "], const T *__restrict__ tab, const int *__restrict__ tcode, unsigned int *hist, "
       "T *Pf, unsigned int *Pi, const T wsT, const unsigned int wsu) {\n";
  std::vector<std::string> v(s.nw), code(s.nb1);
  if (s.ni) {
    if (!fp64) {
      // planar rows: 16-byte part q of row k at plane q, element k (consecutive keys in
      // consecutive bank groups, so a warp's random rows spread over all banks); a tail of one
      // or two words sits in a plane of 4- or 8-byte elements (a random gather of narrower
      // elements takes fewer shared-memory wavefronts)
      static const char *c[4] = {"x", "y", "z", "w"};
      for (int q = 0; q < s.nfull; ++q)
        o << "  const float4 t" << q << " = reinterpret_cast<const float4 *>(tab)[" << (long long)q * s.nkeys
          << " + k];\n";
      const std::string tail = "reinterpret_cast<const " + std::string(s.tew == 4 ? "float4" : s.tew == 2 ? "float2" : "float") +
                               " *>(tab + " + std::to_string((long long)s.nfull * s.nkeys * 4) + ")[k]";
      if (s.tew) o << "  const " << (s.tew == 4 ? "float4" : s.tew == 2 ? "float2" : "float") << " tt = " << tail << ";\n";
      auto word = [&](int p) {
        if (p < 4 * s.nfull) return "t" + std::to_string(p / 4) + "." + c[p % 4];
        return s.tew == 1 ? std::string("tt") : "tt." + std::string(c[p - 4 * s.nfull]);
      };
      for (int w = 0; w < s.nw; ++w) v[w] = word(w);
      for (int b = 0; b < s.nb1; ++b) code[b] = "__float_as_int(" + word(s.nw + b) + ")";
    } else {
      for (int q = 0; q < s.rs / 2; ++q)
        o << "  const double2 t" << q << " = reinterpret_cast<const double2 *>(tab)[" << (long long)q * s.nkeys
          << " + k];\n";
      for (int w = 0; w < s.nw; ++w) v[w] = "t" + std::to_string(w / 2) + (w % 2 ? ".y" : ".x");
      for (int b = 0; b < s.nb1; ++b) code[b] = "tcode[k * " + std::to_string(s.nb1) + " + " + std::to_string(b) + "]";
    }
    o << "  if (" << v[0] << " == (T)0) return;  // no partner in the inner relation\n";
  } else {
    v[0] = "(T)1";
  }
  for (int j = 1; j < s.nm; ++j) o << "  const T u" << j << " = " << basis_expr(s.nx, j) << ";\n";
  for (int j = 0; j < s.nm; ++j)
    for (int w = 0; w < s.nw; ++w) {
      o << "  acc[" << j * s.nw + w << "] += ";
      if (j == 0) o << v[w] << ";\n";
      else o << "u" << j << " * " << v[w] << ";\n";
    }
  if (s.nb1) {
    o << "  const unsigned int cnt = (unsigned int)" << v[0] << ";\n";
    for (int b = 0; b < s.nb1; ++b)
      o << "  { const int c = " << code[b] << "; if (c >= 0) atomicAdd(hist + " << d.b1[b].smem_i << " + c, cnt); }\n";
  }
  for (int c = 0; c < s.n3; ++c) {
    const int pc = d.p3col[c];
    if (d.int3[c]) o << "  atomicAdd(Pi + k * " << s.n3i << " + " << pc << ", wsu);\n";
    else {
      const int j = d.j3[c];
      o << "  atomicAdd(Pf + k * " << s.n3f << " + " << pc << ", wsT" << (j ? " * u" + std::to_string(j) : "")
        << ");\n";
    }
  }
  o << "}\n\n";

  // kernel
  o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", 1) lmfao_gen_root_pass(const GenArgs a) {\n";
  o << "  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n";
  // this CTA's work items: a contiguous range of about 1/G of the tuples, handed to its warps
  // by a ticket in shared memory
  o << "  const Work *__restrict__ work = (const Work *)a.v[" << A_WORK << "];\n";
  o << "  const unsigned long long *__restrict__ wseg = (const unsigned long long *)a.v[" << A_WSEG << "];\n";
  o << "  const int *__restrict__ wq = (const int *)a.v[" << A_WORKQ << "];\n";
  o << "  const int ib = wq[" << kWorkQ << " * blockIdx.x / gridDim.x];\n";
  o << "  const int nwork = wq[" << kWorkQ << " * (blockIdx.x + 1) / gridDim.x];  // end of the range\n";
  o << "  __shared__ unsigned int ticket;\n";
  o << "  const T *__restrict__ gtab = (const T *)a.v[" << A_TABLE << "];\n";
  o << "  const int *__restrict__ gcod = (const int *)a.v[" << A_CODES << "];\n";
  o << "  T *phi0f = (T *)a.v[" << A_PHI0F << "];\n";
  o << "  unsigned long long *phi0i = (unsigned long long *)a.v[" << A_PHI0I << "];\n";
  o << "  unsigned int *phi1i = (unsigned int *)a.v[" << A_PHI1I << "];\n";
  o << "  double *p3f = (double *)a.v[" << A_P3F << "];\n";
  o << "  unsigned long long *p3i = (unsigned long long *)a.v[" << A_P3I << "];\n";
  o << "  const int *__restrict__ kc = (const int *)a.v[" << A_KC << "];\n";
  for (int i = 0; i < s.nx; ++i) {
    if (s.xdt[i] == LMFAO_U8)
      o << "  const unsigned char *__restrict__ xc" << i << " = (const unsigned char *)a.v[" << A_X0 + i << "];\n";
    else
      o << "  const float *__restrict__ xc" << i << " = (const float *)a.v[" << A_X0 + i << "];\n";
  }
  o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
  o << "  T *tab = (T *)(smem + " << s.off_tab << ");\n";
  o << "  int *tcode = (int *)(smem + " << s.off_code << ");\n";
  o << "  T *Pf = (T *)(smem + " << s.off_pf << ");\n";
  o << "  unsigned int *Pi = (unsigned int *)(smem + " << s.off_pi << ");\n";
  o << "  unsigned int *hist0 = (unsigned int *)(smem + " << s.off_h << ");\n";
  o << "  unsigned int *hist = hist0 + warp * " << s.hist << ";\n";
  // staging
  if (s.ni) {
    const int rsw = fp64 ? s.rs : 4 * s.nfull + s.tew;  // staged words per row
    o << "#pragma unroll 4\n";  // several loads of the staging loop in flight
    o << "  for (int i = tid; i < " << s.nkeys * rsw << "; i += " << block << ") {\n";
    o << "    const int k = i / " << rsw << ", c = i - k * " << rsw << ";\n";
    o << "    T t = (T)0;\n";
    o << "    if (c < " << s.nw << ") t = gtab[(long long)k * " << s.nw << " + c];\n";
    if (!fp64)
      for (int b = 0; b < s.nb1; ++b)
        o << "    else if (c == " << s.nw + b << ") t = __int_as_float(gcod[(long long)k * " << s.ncode << " + "
          << d.b1code[b] << "]);\n";
    if (fp64) {
      o << "    tab[(c / 2) * " << s.nkeys * 2 << " + k * 2 + c % 2] = t;\n  }\n";
    } else {
      o << "    if (c < " << 4 * s.nfull << ") tab[(c / 4) * " << s.nkeys * 4 << " + k * 4 + c % 4] = t;\n";
      o << "    else tab[" << (long long)s.nfull * s.nkeys * 4 << " + k * " << s.tew << " + c - " << 4 * s.nfull
        << "] = t;\n  }\n";
    }
    if (fp64 && s.nb1) {
      o << "  for (int i = tid; i < " << s.nkeys * s.nb1 << "; i += " << block << ") {\n";
      o << "    const int k = i / " << s.nb1 << ", b = i - k * " << s.nb1 << ";\n";
      o << "    int c = -1;\n";
      for (int b = 0; b < s.nb1; ++b)
        o << "    if (b == " << b << ") c = gcod[(long long)k * " << s.ncode << " + " << d.b1code[b] << "];\n";
      o << "    tcode[i] = c;\n  }\n";
    }
  }
  o << "  for (int i = tid; i < " << s.nkeys * s.n3f << "; i += " << block << ") Pf[i] = (T)0;\n";
  o << "  for (int i = tid; i < " << s.nkeys * s.n3i << "; i += " << block << ") Pi[i] = 0u;\n";
  o << "  for (int i = tid; i < " << (long long)(block / 32) * s.hist << "; i += " << block << ") hist0[i] = 0u;\n";
  o << "  if (tid == 0) ticket = 0u;\n";
  o << "  __syncthreads();\n";
  // work loop: the ticket, record and outer weight of the next work item and the first quad
  // of each lane in it are requested while the current item is processed
  auto scalar_x = [&](int i) { return "(T)xc" + std::to_string(i) + "[r]"; };
  auto xreg_type = [&](int i) { return s.xdt[i] == LMFAO_U8 ? std::string("unsigned int") : std::string("float4"); };
  auto xreg_load = [&](int i, const std::string &q) {
    if (s.xdt[i] == LMFAO_U8) return "reinterpret_cast<const unsigned int *>(xc" + std::to_string(i) + ")[" + q + "]";
    return "reinterpret_cast<const float4 *>(xc" + std::to_string(i) + ")[" + q + "]";
  };
  auto quad_load = [&](const std::string &q, const std::string &ind) {
    if (s.ni) o << ind << "kn = reinterpret_cast<const int4 *>(kc)[" << q << "];\n";
    for (int i = 0; i < s.nx; ++i) o << ind << "xn" << i << " = " << xreg_load(i, q) << ";\n";
  };
  o << "  int wi;\n";
  o << "  {\n    unsigned int t = 0u;\n    if (lane == 0) t = atomicAdd(&ticket, 1u);\n";
  o << "    wi = ib + (int)__shfl_sync(0xffffffffu, t, 0);\n  }\n";
  o << "  Work wk = {0, 0, 0};\n  unsigned long long ws = 0ull;\n";
  o << "  if (wi < nwork) { wk = work[wi]; ws = wseg[wk.seg]; }\n";
  if (d.lanes) {
    // one tuple per lane and step: tuple r0 + lane + 32 i; the next step's key and values are
    // loaded while the current tuple is processed (coalesced 4-byte loads, no ragged edges)
    // a ring of D steps in flight per lane: slot j holds tuple r + 32 j
    const int D = 4;
    auto lane_load_slot = [&](int j, const std::string &r, const std::string &ind) {
      if (s.ni) o << ind << "kn" << j << " = kc[" << r << "];\n";
      for (int i = 0; i < s.nx; ++i) o << ind << "xn" << i << "_" << j << " = (T)xc" << i << "[" << r << "];\n";
    };
    auto lane_fill = [&](const std::string &base, const std::string &end, const std::string &ind) {
      for (int j = 0; j < D; ++j) {
        o << ind << "if (" << base << " + " << 32 * j << " < " << end << ") {\n";
        lane_load_slot(j, base + " + " + std::to_string(32 * j), ind + "  ");
        o << ind << "}\n";
      }
    };
    for (int j = 0; j < D; ++j) {
      if (s.ni) o << "  int kn" << j << " = 0;\n";
      for (int i = 0; i < s.nx; ++i) o << "  T xn" << i << "_" << j << " = (T)0;\n";
    }
    o << "  long long r = wk.r0 + lane;\n";
    lane_fill("r", "wk.r0 + wk.len", "  ");
    o << "  while (wi < nwork) {\n";
    o << "    int wn;  // the next item (shared-memory ticket): its record is requested now\n";
    o << "    {\n      unsigned int t = 0u;\n      if (lane == 0) t = atomicAdd(&ticket, 1u);\n";
    o << "      wn = ib + (int)__shfl_sync(0xffffffffu, t, 0);\n    }\n";
    o << "    Work wkn = {0, 0, 0};\n";
    o << "    if (wn < nwork) wkn = work[wn];  // used after the tuples of this item\n";
    o << "    const T wsT = (T)ws;\n";
    o << "    const unsigned int wsu = (unsigned int)ws;\n";
    o << "    T acc[" << V << "];\n";
    o << "#pragma unroll\n    for (int i = 0; i < " << V << "; ++i) acc[i] = (T)0;\n";
    o << "    if (ws != 0ull) {  // else no outer partner for the whole segment\n";
    o << "      const long long rend = wk.r0 + wk.len;\n";
    // D steps per iteration: slot j is consumed and refilled with the tuple D steps ahead, so
    // every slot's load has a whole iteration to land (no register moves between slots)
    auto lane_tuple = [&](int j, const std::string &ind) {
      o << ind << "tuple(" << (s.ni ? "kk" : "0");
      for (int i = 0; i < 3; ++i) o << ", " << (i < s.nx ? "xk" + std::to_string(i) : std::string("(T)0"));
      o << ", acc, tab, tcode, hist, Pf, Pi, wsT, wsu);\n";
      (void)j;
    };
    o << "      for (; r + " << 32 * (D - 1) << " < rend; r += " << 32 * D << ") {\n";
    for (int j = 0; j < D; ++j) {
      o << "        {\n";
      if (s.ni) o << "          const int kk = kn" << j << ";\n";
      for (int i = 0; i < s.nx; ++i) o << "          const T xk" << i << " = xn" << i << "_" << j << ";\n";
      o << "          if (r + " << 32 * (D + j) << " < rend) {\n";
      lane_load_slot(j, "r + " + std::to_string(32 * (D + j)), "            ");
      o << "          }\n";
      lane_tuple(j, "          ");
      o << "        }\n";
    }
    o << "      }\n";
    // the last steps of the item (fewer than D), already in the slots
    for (int j = 0; j + 1 < D; ++j) {
      o << "      if (r + " << 32 * j << " < rend) {\n";
      if (s.ni) o << "        const int kk = kn" << j << ";\n";
      for (int i = 0; i < s.nx; ++i) o << "        const T xk" << i << " = xn" << i << "_" << j << ";\n";
      lane_tuple(j, "        ");
      o << "      }\n";
    }
    o << "    }\n";
    o << "    unsigned long long wsn = 0ull;\n";
    o << "    if (wn < nwork) wsn = wseg[wkn.seg];\n";
    o << "    r = wkn.r0 + lane;\n";
    lane_fill("r", "wkn.r0 + wkn.len", "    ");
  } else {
  o << "  long long qa = (wk.r0 + 3) >> 2, qe = (wk.r0 + wk.len) >> 2;\n";
  o << "  if (qe < qa) qe = qa;\n";
  if (s.ni) o << "  int4 kn = make_int4(0, 0, 0, 0);\n";
  for (int i = 0; i < s.nx; ++i) o << "  " << xreg_type(i) << " xn" << i << "{};\n";
  o << "  long long q = qa + lane;\n";
  o << "  if (q < qe) {\n";
  quad_load("q", "    ");
  o << "  }\n";
  o << "  while (wi < nwork) {\n";
  o << "    int wn;  // the next item (shared-memory ticket): its record is requested now\n";
  o << "    {\n      unsigned int t = 0u;\n      if (lane == 0) t = atomicAdd(&ticket, 1u);\n";
  o << "      wn = ib + (int)__shfl_sync(0xffffffffu, t, 0);\n    }\n";
  o << "    Work wkn = {0, 0, 0};\n";
  o << "    if (wn < nwork) wkn = work[wn];  // used after the tuples of this item\n";
  o << "    const T wsT = (T)ws;\n";
  o << "    const unsigned int wsu = (unsigned int)ws;\n";
  o << "    T acc[" << V << "];\n";
  o << "#pragma unroll\n    for (int i = 0; i < " << V << "; ++i) acc[i] = (T)0;\n";
  o << "    if (ws != 0ull) {  // else no outer partner for the whole segment\n";
  o << "      const long long r0 = wk.r0, rend = r0 + wk.len;\n";
  o << "      const long long he = 4 * qa < rend ? 4 * qa : rend;\n";
  o << "      const long long te = 4 * qe > he ? 4 * qe : he;\n";
  // ragged head and tail
  o << "      {\n        long long r = -1;\n";
  o << "        if (lane < 4) { if (r0 + lane < he) r = r0 + lane; }\n";
  o << "        else if (lane >= 8 && lane < 12) { if (te + (lane - 8) < rend) r = te + (lane - 8); }\n";
  o << "        if (r >= 0) tuple(" << (s.ni ? "kc[r]" : "0");
  for (int i = 0; i < 3; ++i) o << ", " << (i < s.nx ? scalar_x(i) : std::string("(T)0"));
  o << ", acc, tab, tcode, hist, Pf, Pi, wsT, wsu);\n      }\n";
  // full quads with the next quad in flight
  o << "      for (; q < qe; q += 32) {\n";
  if (s.ni) o << "        const int4 kk = kn;\n";
  for (int i = 0; i < s.nx; ++i) o << "        const " << xreg_type(i) << " xk" << i << " = xn" << i << ";\n";
  o << "        if (q + 32 < qe) {\n";
  quad_load("q + 32", "          ");
  o << "        }\n";
  static const char *comp[4] = {"x", "y", "z", "w"};
  for (int u = 0; u < 4; ++u) {
    o << "        tuple(" << (s.ni ? std::string("kk.") + comp[u] : std::string("0"));
    for (int i = 0; i < 3; ++i) o << ", " << (i < s.nx ? x_component(s.xdt[i], "xk" + std::to_string(i), u) : "(T)0");
    o << ", acc, tab, tcode, hist, Pf, Pi, wsT, wsu);\n";
  }
  o << "      }\n    }\n";
  // the next item: its weight and first quad overlap with the segment sums of this one
  o << "    unsigned long long wsn = 0ull;\n";
  o << "    if (wn < nwork) wsn = wseg[wkn.seg];\n";
  o << "    long long qan = (wkn.r0 + 3) >> 2, qen = (wkn.r0 + wkn.len) >> 2;\n";
  o << "    if (qen < qan) qen = qan;\n";
  o << "    q = qan + lane;\n";
  o << "    if (q < qen) {\n";
  quad_load("q", "      ");
  o << "    }\n";
  }
  o << "    if (ws != 0ull) {\n";
  // per-segment sums: reduce-scatter over the warp
  const WarpReduce wr = gen_warp_reduce(V, "    ");
  o << wr.src;
  o << gen_reduce_flush(wr, "phi0f", "(long long)wk.seg * " + std::to_string(V), "    ");
  if (s.n0i) {
    o << "    {\n      T iv = (T)0;\n";
    for (int e = 0; e < s.n0i; ++e) {
      const int q = d.i0j[e] * s.nw + d.i0w[e];
      o << "      { const T t = __shfl_sync(0xffffffffu, r_[" << wr.reg_of(q) << "], " << wr.lane_of(q)
        << "); if (lane == " << e << ") iv = t; }\n";
    }
    o << "      if (lane < " << s.n0i << ") {\n";
    o << "        const unsigned long long it = (unsigned long long)(iv + (T)0.5);\n";
    o << "        if (it) atomicAdd(phi0i + (long long)wk.seg * " << s.n0i << " + lane, it);\n      }\n    }\n";
  }
  if (s.nb1) {
    o << "    __syncwarp();\n";
    for (int b = 0; b < s.nb1; ++b) {
      o << "    for (int i = lane; i < " << d.b1[b].G << "; i += 32) {\n";
      o << "      const unsigned int x = hist[" << d.b1[b].smem_i << " + i];\n";
      o << "      if (x) { hist[" << d.b1[b].smem_i << " + i] = 0u; atomicAdd(phi1i + (long long)wk.seg * "
        << s.phi1i_seg << " + " << d.b1[b].gbase_i << " + i, x); }\n    }\n";
    }
    o << "    __syncwarp();\n";
  }
  o << "    }\n";
  if (d.lanes) o << "    wi = wn;\n    wk = wkn;\n    ws = wsn;\n";
  else o << "    wi = wn;\n    wk = wkn;\n    ws = wsn;\n    qa = qan;\n    qe = qen;\n";
  o << "  }\n";
  // root-to-inner partials: CTA-private -> global
  o << "  __syncthreads();\n";
  o << "  for (int i = tid; i < " << s.nkeys * s.n3f << "; i += " << block
    << ") if (Pf[i] != (T)0) atomicAdd(p3f + i, (double)Pf[i]);\n";
  o << "  for (int i = tid; i < " << s.nkeys * s.n3i << "; i += " << block
    << ") if (Pi[i]) atomicAdd(p3i + i, (unsigned long long)Pi[i]);\n";
  o << "}\n";
  return o.str();
}

namespace {

struct Compiled {
  const void *fn = nullptr;
  std::string err;
};

std::mutex cache_mu;
std::map<std::string, Compiled> cache;  // by source text (the device is the same sm_103a part)

Compiled compile(const std::string &src, const char *name = "lmfao_gen_root_pass") {
  Compiled c;
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "lmfao_gen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    c.err = "nvrtcCreateProgram failed";
    return c;
  }
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo"};
  nvrtcResult r = nvrtcCompileProgram(prog, 3, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    c.err = std::string("NVRTC: ") + nvrtcGetErrorString(r) + ": " + log.substr(0, 400);
    nvrtcDestroyProgram(&prog);
    return c;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  std::string cubin(n, '\0');
  nvrtcGetCUBIN(prog, &cubin[0]);
  nvrtcDestroyProgram(&prog);
  cudaLibrary_t lib;
  if (cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
    cudaGetLastError();
    c.err = "cudaLibraryLoadData failed";
    return c;
  }
  cudaKernel_t k;
  if (cudaLibraryGetKernel(&k, lib, name) != cudaSuccess) {
    cudaGetLastError();
    c.err = "cudaLibraryGetKernel failed";
    return c;
  }
  c.fn = (const void *)k;
  return c;
}

bool eligible(const DFast &d, std::string &why) {
  if (!d.lean) why = "not a lean root pass";
  else if (!d.vec) why = "root columns not reorganised (no vector loads)";
  else if (d.ni && d.nk != 1) why = "inner key of more than one attribute";
  else if (d.nfam || d.nb4) why = "filter family";
  else if (d.nx > 3) why = "more than 3 value columns";
  else if (!d.ni && (d.nb1 || d.n3 || d.nw != 1)) why = "inner items without an inner relation";
  else if (d.nm != 1 + d.nx + d.nx * (d.nx + 1) / 2) why = "monomials are not the degree <= 2 basis";
  if (!why.empty()) return false;
  for (int i = 0; i < d.nx; ++i) {
    const int dt = d.col[d.xslot[i]].dtype;
    if (dt != LMFAO_F32 && dt != LMFAO_U8) {
      why = "value column type";
      return false;
    }
  }
  if (d.ni && d.col[d.kslot[0]].dtype != LMFAO_I32) {
    why = "inner key type";
    return false;
  }
  return true;
}

}  // namespace

namespace {

// compile (or take from the cache) and check one generated source
std::string fnv1a_hex(const std::string &text) {
  unsigned long long h = 1469598103934665603ull;
  for (unsigned char ch : text) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  char buf[17];
  snprintf(buf, sizeof buf, "%016llx", h);
  return buf;
}

bool finish(GenRootPass &g, const std::string &src, int block, size_t smem) {
  g.source_hash = fnv1a_hex(src);
  Compiled c;
  {
    std::lock_guard<std::mutex> lk(cache_mu);
    auto it = cache.find(src);
    if (it != cache.end()) c = it->second;
    else {
      c = compile(src);
      cache[src] = c;
    }
  }
  if (!c.fn) {
    g.why = c.err;
    return false;
  }
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, c.fn) != cudaSuccess) {
    cudaGetLastError();
    g.why = "cudaFuncGetAttributes failed";
    return false;
  }
  if (fa.localSizeBytes > 0 && block > 512) {
    g.why = "register spills";
    return false;
  }
  if (cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    g.why = "shared memory attribute";
    return false;
  }
  g.fn = c.fn;
  g.block = block;
  g.smem = smem;
  g.why.clear();
  return true;
}

GenRootPass gen_family(const DFast &d, bool fp64, const std::vector<float> &thr) {
  GenRootPass g;
  g.family = true;
  // host copies of the CTA-private items' group references and output regions
  int nref4 = 0;
  for (int i = 0; i < d.nb4; ++i) nref4 = std::max(nref4, d.b4_g0[i] + d.b4_ng[i]);
  std::vector<DGroupRef> grefs4(nref4);
  std::vector<DMirror> mirror(d.nb4mirror);
  if ((nref4 && cudaMemcpy(grefs4.data(), d.grefs4, nref4 * sizeof(DGroupRef), cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (d.nb4mirror &&
       cudaMemcpy(mirror.data(), d.b4mirror, d.nb4mirror * sizeof(DMirror), cudaMemcpyDeviceToHost) != cudaSuccess)) {
    cudaGetLastError();
    g.why = "descriptor copy failed";
    return g;
  }
  if (!family_eligible(d, g.why, grefs4)) return g;
  for (int block : {fp64 ? 512 : 1024, 512}) {
    const FamilyLayout L = family_layout(d, fp64, block);
    if (L.smem > 227 * 1024) {
      g.why = "shared memory";
      continue;
    }
    if (finish(g, gen_family_source(d, fp64, block, thr, grefs4, mirror), block, L.smem)) return g;
    if (g.why != "register spills") return g;
  }
  return g;
}

}  // namespace

GenRootPass gen_root_pass(const DFast &d, bool fp64, int device, const std::vector<float> &thr) {
  (void)device;
  if (!d.lean || d.nfam || d.nb4) return gen_family(d, fp64, thr);
  GenRootPass g;
  if (!eligible(d, g.why)) return g;
  for (int block : {fp64 ? 512 : 1024, 512}) {
    const Shape s = shape_of(d, fp64, block);
    if (s.smem > 227 * 1024) {
      g.why = "shared memory";
      continue;
    }
    if (finish(g, gen_root_pass_source(d, fp64, block), block, s.smem)) return g;
    if (g.why != "register spills") return g;
  }
  return g;
}

cudaError_t launch_gen_root_pass(const GenRootPass &g, const DFast &d, int grid, cudaStream_t s) {
  GenArgs a{};
  a.v[A_NWORK] = (unsigned long long)d.nwork;
  a.v[A_WORK] = (unsigned long long)d.work;
  a.v[A_WSEG] = (unsigned long long)d.wseg;
  a.v[A_WORKQ] = (unsigned long long)d.work_q;
  a.v[A_TABLE] = (unsigned long long)d.table;
  a.v[A_CODES] = (unsigned long long)d.codes;
  a.v[A_PHI0F] = (unsigned long long)d.phi0f;
  a.v[A_PHI0I] = (unsigned long long)d.phi0i;
  a.v[A_PHI1I] = (unsigned long long)d.phi1i;
  a.v[A_P3F] = (unsigned long long)d.p3f;
  a.v[A_P3I] = (unsigned long long)d.p3i;
  a.v[A_KC] = d.ni ? (unsigned long long)d.col[d.kslot[0]].p : 0ull;
  for (int i = 0; i < d.nx && i < 3; ++i) a.v[A_X0 + i] = (unsigned long long)d.col[d.xslot[i]].p;
  void *args[] = {&a};
  if (!g.family) return cudaLaunchKernel(g.fn, dim3(grid), dim3(g.block), args, g.smem, s);
  struct { unsigned long long v[32]; } f{};
  f.v[F_NWORK] = (unsigned long long)d.nwork;
  f.v[F_WORK] = (unsigned long long)d.work;
  f.v[F_WSEG] = (unsigned long long)d.wseg;
  f.v[F_WORKQ] = (unsigned long long)d.work_q;
  f.v[F_TABLE] = (unsigned long long)d.table;
  f.v[F_CODES] = (unsigned long long)d.codes;
  f.v[F_PHI0F] = (unsigned long long)d.phi0f;
  f.v[F_PHI0I] = (unsigned long long)d.phi0i;
  f.v[F_PHI1F] = (unsigned long long)d.phi1f;
  f.v[F_PHI1I] = (unsigned long long)d.phi1i;
  f.v[F_P3F] = (unsigned long long)d.p3f;
  f.v[F_P3F32] = (unsigned long long)d.p3f32;
  f.v[F_P3I] = (unsigned long long)d.p3i;
  f.v[F_FSUM] = (unsigned long long)d.fsum;
  f.v[F_ICNT] = (unsigned long long)d.icnt;
  f.v[F_KC] = d.ni ? (unsigned long long)d.col[d.kslot[0]].p : 0ull;
  for (int i = 0; i < d.nx && i < 6; ++i) f.v[F_X0 + i] = (unsigned long long)d.col[d.xslot[i]].p;
  // outer views of the predicate bits, in the order the generator assigned their slots
  int used[MAXOUT] = {0}, nov = 0;
  for (int b = 0; b < (d.nfam ? d.nob : 0); ++b) {
    const int ov = d.obit_outer[b];
    bool seen = false;
    for (int j = 0; j < nov; ++j) seen = seen || used[j] == ov;
    if (!seen && nov < 6) {
      used[nov] = ov;
      f.v[F_OV0 + nov] = (unsigned long long)d.outer[ov].v.v64;
      ++nov;
    }
  }
  void *fargs[] = {&f};
  return cudaLaunchKernel(g.fn, dim3(grid), dim3(g.block), fargs, g.smem, s);
}


// ------------------------------------------------------------------ generated view kernel
// The view of a relation with unique keys and no children (view_key_rows_kernel's job) with
// the columns as straight-line code: one thread per key reads the row's input columns into
// registers once, forms every column (product of its factors, left to right as fac_at does,
// times 1 or 0 for the row's presence) and its codes, into a shared tile written out by the
// CTA as one contiguous span.
namespace {
const char *cmp_text(int op) {
  switch (op) {
    case LMFAO_LE: return "<=";
    case LMFAO_LT: return "<";
    case LMFAO_GE: return ">=";
    case LMFAO_GT: return ">";
    case LMFAO_EQ: return "==";
    default: return "!=";
  }
}
std::string flt_lit(float t) {
  std::ostringstream o;
  o.precision(9);
  o << std::scientific << t << "f";
  return o.str();
}
}  // namespace

std::string gen_view_source(const DViewKernel &d, const std::vector<int> &cfo, const std::vector<DFac> &facs,
                            const std::vector<int4> &cdesc, const std::vector<float> &thr) {
  const int W = d.ncols + 1, KB = kVkb;
  std::ostringstream o;
  o << "// generated view kernel\n";
  o << "struct GenArgs { unsigned long long v[32]; };\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << KB << ") lmfao_gen_view(const GenArgs a) {\n";
  o << "  __shared__ double tile[" << KB * W << "];\n";
  o << "  const long long nkeys = (long long)a.v[0];\n";
  o << "  const int *__restrict__ keyrow = (const int *)a.v[1];\n";
  o << "  double *v64 = (double *)a.v[2];\n";
  o << "  int *codes = (int *)a.v[3];\n";
  std::vector<bool> used(d.ncolsin, false);
  for (const DFac &f : facs) used[f.col] = true;
  for (const int4 &c : cdesc) used[c.x] = true;
  auto ctype = [&](int slot) {
    return d.in[slot].dtype == LMFAO_F32 ? "float" : d.in[slot].dtype == LMFAO_U8 ? "unsigned char" : "int";
  };
  for (int i = 0; i < d.ncolsin; ++i)
    if (used[i]) o << "  const " << ctype(i) << " *__restrict__ c" << i << " = (const " << ctype(i) << " *)a.v[" << 4 + i << "];\n";
  o << "  const int t = threadIdx.x;\n";
  o << "  const long long k0 = (long long)blockIdx.x * " << KB << ";\n";
  o << "  const int nk = (int)(nkeys - k0 < " << KB << " ? nkeys - k0 : " << KB << ");\n";
  o << "  if (t < nk) {\n";
  o << "    const long long k = k0 + t;\n";
  o << "    const int r = keyrow[k];\n";
  o << "    const bool live = r >= 0;\n";
  o << "    const int rr = live ? r : 0;\n";
  for (int i = 0; i < d.ncolsin; ++i)
    if (used[i]) o << "    const " << ctype(i) << " x" << i << " = c" << i << "[rr];\n";
  o << "    const double lv = live ? 1.0 : 0.0;\n";
  for (int j = 0; j < d.ncols; ++j) {
    std::string e = "lv";
    for (int f = cfo[j]; f < cfo[j + 1]; ++f) {
      const DFac &fc = facs[f];
      std::string term;
      if (fc.ind) {
        // predicates compare the stored value: FP32 columns in FP32, integer columns exactly
        const std::string x = "x" + std::to_string(fc.col);
        term = d.in[fc.col].dtype == LMFAO_F32 ? "(" + x + " " + cmp_text(fc.op) + " " + flt_lit(fc.t) + " ? 1.0 : 0.0)"
                                              : "((double)" + x + " " + cmp_text(fc.op) + " (double)" + flt_lit(fc.t) + " ? 1.0 : 0.0)";
      } else {
        const std::string x = "(double)x" + std::to_string(fc.col);
        term = x;
        for (int p = 1; p < fc.pow; ++p) term = "(" + term + " * " + x + ")";
      }
      e = "(" + e + " * " + term + ")";
    }
    o << "    tile[t * " << W << " + " << j << "] = " << e << ";\n";
  }
  for (size_t c = 0; c < cdesc.size(); ++c) {
    const int4 cd = cdesc[c];
    std::string code;
    if (cd.y == LMFAO_GB_BUCKET) {
      const std::string xf = "(float)x" + std::to_string(cd.x);
      code = "0";
      for (int q = 0; q < cd.w; ++q) code += " + (" + flt_lit(thr[cd.z + q]) + " < " + xf + ")";
    } else {
      code = "(int)x" + std::to_string(cd.x);
    }
    o << "    codes[k * " << cdesc.size() << " + " << c << "] = live ? (" << code << ") : -1;\n";
  }
  o << "  }\n";
  o << "  __syncthreads();\n";
  o << "  const int lane = t & 31, warp = t >> 5;\n";
  o << "  double *out = v64 + k0 * " << d.ncols << ";\n";
  o << "  for (int q = warp; q < nk; q += " << KB / 32 << ")\n";
  o << "    for (int j = lane; j < " << d.ncols << "; j += 32) out[(long long)q * " << d.ncols << " + j] = tile[q * " << W
    << " + j];\n";
  o << "}\n";
  return o.str();
}

GenView gen_view(const DViewKernel &d, const std::vector<int> &cfo, const std::vector<DFac> &facs,
                 const std::vector<int4> &cdesc, const std::vector<float> &thr) {
  GenView g;
  if (!d.keyrow) g.why = "keys not unique or key tile too large";
  else if (d.nchild) g.why = "relation with children";
  else if (d.ncolsin > 28) g.why = "more than 28 input columns";
  else if (d.ncols > 64) g.why = "more than 64 columns";
  for (const int4 &c : cdesc)
    if (c.x < 0) g.why = "code from a child";
  if (!g.why.empty()) return g;
  const std::string src = gen_view_source(d, cfo, facs, cdesc, thr);
  g.source_hash = fnv1a_hex(src);
  Compiled c;
  {
    std::lock_guard<std::mutex> lk(cache_mu);
    auto it = cache.find(src);
    if (it != cache.end()) c = it->second;
    else {
      c = compile(src, "lmfao_gen_view");
      cache[src] = c;
    }
  }
  if (!c.fn) g.why = c.err;
  g.fn = c.fn;
  return g;
}

cudaError_t launch_gen_view(const GenView &g, const DViewKernel &d, cudaStream_t s) {
  if (d.nkeys == 0) return cudaSuccess;
  struct { unsigned long long v[32]; } a{};
  a.v[0] = (unsigned long long)d.nkeys;
  a.v[1] = (unsigned long long)d.keyrow;
  a.v[2] = (unsigned long long)d.v64;
  a.v[3] = (unsigned long long)d.codes;
  for (int i = 0; i < d.ncolsin && i < 28; ++i) a.v[4 + i] = (unsigned long long)d.in[i].p;
  void *args[] = {&a};
  return cudaLaunchKernel(g.fn, dim3((unsigned)((d.nkeys + kVkb - 1) / kVkb)), dim3(kVkb), args, 0, s);
}

}  // namespace lmfao
