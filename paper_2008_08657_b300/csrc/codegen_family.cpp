// Plan-specialised root pass for the general specialised shape (any monomials over the root's
// value columns, indicator factors, a filter family such as the leaves of a decision-tree
// level, leaf-split root-to-inner partials and CTA-private items), generated as CUDA source
// and compiled with NVRTC like the lean pass of codegen.cpp.
//
// The generated kernel computes what fast_pass_kernel computes for the same DFast, with every
// descriptor folded into constants: the monomials as products of powers of the tuple's value
// columns, the predicate bits of the tuple's filter (outer bits once per segment, inner bits
// from the inner row, root bits per tuple) and its leaf, bucket codes of root columns as
// comparisons against the constant thresholds (once per tuple and column), and the scatter of
// each histogram set, root-to-inner column and CTA-private item with constant offsets. The
// integral root-to-inner partials stay in shared memory when they fit even if the float ones
// do not (a decision-tree level: 3,700 items x 8 leaves), which removes one global atomic per
// tuple and column.
#include <cuda_runtime.h>

#include <map>
#include <sstream>

#include "codegen.h"

namespace lmfao {

namespace {

int rup(int x, int m) { return (x + m - 1) / m * m; }

const char *cmp_src(int op) {
  switch (op) {
    case LMFAO_LE: return "<=";
    case LMFAO_LT: return "<";
    case LMFAO_GE: return ">=";
    case LMFAO_GT: return ">";
    case LMFAO_EQ: return "==";
    default: return "!=";
  }
}

std::string flt(float t) {
  std::ostringstream o;
  o.precision(9);
  o << std::scientific << t << "f";
  return o.str();
}

}  // namespace

FamilyLayout family_layout(const DFast &d, bool fp64, int block) {
  FamilyLayout L{};
  const int nw = d.ni ? d.nw : 1;
  const size_t ts = fp64 ? 8 : 4;
  const long long nkeys = d.ni ? d.nkeys : 0;
  L.rs = fp64 ? rup(nw, 2) : rup(nw + d.ncode, 4);
  L.nfull = (nw + d.ncode) / 4;
  L.tew = (nw + d.ncode) % 4 == 3 ? 4 : (nw + d.ncode) % 4;  // a tail of 1 or 2 words: 4- or 8-byte loads
  size_t off = 0;
  auto region = [&](size_t bytes) {
    size_t at = off;
    off = (off + bytes + 15) & ~(size_t)15;
    return at;
  };
  const int ls = std::max(1, d.b3leaf);
  const size_t pi_bytes = 4 * (size_t)nkeys * d.n3i * ls;
  for (int pass = 0; pass < 2; ++pass) {
    // first try the integral partials in shared memory even when the float ones do not fit
    L.pi_smem = d.smem_p || (pass == 0 && d.n3i > 0);
    off = 0;
    L.off_tab = region(fp64 ? ts * (size_t)nkeys * L.rs : 4 * (size_t)nkeys * (4 * L.nfull + L.tew));
    L.off_code = region(fp64 ? 4 * (size_t)nkeys * d.ncode : 0);
    L.off_pf = region(d.smem_p ? ts * (size_t)nkeys * d.n3f * ls : 0);
    L.off_pi = region(L.pi_smem ? pi_bytes : 0);
    L.off_h = region(4 * (size_t)(block / 32) * (d.hist_f + d.hist_i));
    L.off_b4f = region(ts * (size_t)d.b4_fcells);
    L.off_b4i = region(4 * (size_t)d.b4_icells);
    L.smem = off;
    if (d.smem_p || !L.pi_smem || L.smem <= 200 * 1024) break;
  }
  return L;
}

bool family_eligible(const DFast &d, std::string &why, const std::vector<DGroupRef> &grefs4) {
  auto xidx = [&](int slot) {
    for (int i = 0; i < d.nx; ++i)
      if (d.xslot[i] == slot) return i;
    return -1;
  };
  if (!d.vec) why = "root columns not reorganised (no vector loads)";
  else if (d.ni && d.nk != 1) why = "inner key of more than one attribute";
  else if (d.nx > 6) why = "more than 6 value columns";
  else if (!d.ni && (d.nb1 || d.n3)) why = "inner items without an inner relation";
  if (!why.empty()) return false;
  for (int i = 0; i < d.nx; ++i) {
    const int dt = d.col[d.xslot[i]].dtype;
    if (dt != LMFAO_F32 && dt != LMFAO_U8) { why = "value column type"; return false; }
  }
  if (d.ni && d.col[d.kslot[0]].dtype != LMFAO_I32) { why = "inner key type"; return false; }
  for (int f = 0; f < d.nind; ++f)
    if (xidx(d.ind[f].col) < 0) { why = "indicator on a column that is not a value column"; return false; }
  for (int q = 0; q < d.nrb; ++q)
    if (xidx(d.rb[q].col) < 0) { why = "root predicate on a column that is not a value column"; return false; }
  auto ref_ok = [&](const DGroupRef &q) {
    if (q.src == 2) return xidx(q.a) >= 0 && q.kind == LMFAO_GB_BUCKET;
    return q.src == 3 || q.src == 4;
  };
  for (int s = 0; s < d.nb1; ++s)
    for (int i = 0; i < d.b1[s].nref; ++i)
      if (!ref_ok(d.b1[s].ref[i])) { why = "histogram group code"; return false; }
  for (const DGroupRef &q : grefs4)
    if ((q.src != 2 && q.src != 3) || !ref_ok(q)) { why = "CTA-private item group code"; return false; }
  return true;
}

std::string gen_family_source(const DFast &d, bool fp64, int block, const std::vector<float> &thr,
                              const std::vector<DGroupRef> &grefs4, const std::vector<DMirror> &mirror) {
  const FamilyLayout L = family_layout(d, fp64, block);
  const int nw = d.ni ? d.nw : 1, nm = d.nm, nx = d.nx;
  const long long nkeys = d.ni ? d.nkeys : 0;
  const int V = nm * nw;
  // Histogram sets with few cells (such as one per leaf of a decision-tree level) are kept in
  // registers: their float cells extend the per-lane segment sums acc[] (reduced over the warp
  // with them), their integral cells sit in hri[] (summed with the warp's integer reduction).
  // Every tuple of a warp then adds to registers instead of a few shared-memory cells that the
  // whole warp would hit with serialised atomics.
  std::vector<int> hoff(d.nb1, -1), hoffi(d.nb1, -1);
  int VX = V, NRI = 0;
  if (V <= 32)
    for (int s = 0; s < d.nb1; ++s) {
      const DFastB1 &b = d.b1[s];
      if (b.G <= 8 && VX + b.G * b.nf <= 32 && NRI + b.G * b.ni <= 8) {
        hoff[s] = VX;
        hoffi[s] = NRI;
        VX += b.G * b.nf;
        NRI += b.G * b.ni;
      }
    }
  const int ls = std::max(1, d.b3leaf);
  auto xidx = [&](int slot) {
    for (int i = 0; i < nx; ++i)
      if (d.xslot[i] == slot) return i;
    return -1;
  };
  std::ostringstream o;
  o << "// generated root pass (filter family)\n";
  o << "typedef " << (fp64 ? "double" : "float") << " T;\n";
  o << "struct GenArgs { unsigned long long v[32]; };\n";
  o << "struct Work { long long r0; int seg; int len; };\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << block << ", 1) lmfao_gen_root_pass(const GenArgs a) {\n";
  o << "  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n";
  // this CTA's work items (a contiguous range of about 1/G of the tuples) and its ticket
  o << "  const Work *__restrict__ work = (const Work *)a.v[" << F_WORK << "];\n";
  o << "  const unsigned long long *__restrict__ wseg = (const unsigned long long *)a.v[" << F_WSEG << "];\n";
  o << "  const int *__restrict__ wq = (const int *)a.v[" << F_WORKQ << "];\n";
  o << "  const int ib = wq[" << kWorkQ << " * blockIdx.x / gridDim.x];\n";
  o << "  const int nwork = wq[" << kWorkQ << " * (blockIdx.x + 1) / gridDim.x];  // end of the range\n";
  o << "  __shared__ unsigned int ticket;\n";
  o << "  const T *__restrict__ gtab = (const T *)a.v[" << F_TABLE << "];\n";
  o << "  const int *__restrict__ gcod = (const int *)a.v[" << F_CODES << "];\n";
  o << "  T *phi0f = (T *)a.v[" << F_PHI0F << "];\n";
  o << "  unsigned long long *phi0i = (unsigned long long *)a.v[" << F_PHI0I << "];\n";
  o << "  float *phi1f = (float *)a.v[" << F_PHI1F << "];\n";
  o << "  unsigned int *phi1i = (unsigned int *)a.v[" << F_PHI1I << "];\n";
  o << "  double *p3f = (double *)a.v[" << F_P3F << "];\n";
  o << "  float *p3f32 = (float *)a.v[" << F_P3F32 << "];\n";
  o << "  unsigned long long *p3i = (unsigned long long *)a.v[" << F_P3I << "];\n";
  o << "  double *fsum = (double *)a.v[" << F_FSUM << "];\n";
  o << "  unsigned long long *icnt = (unsigned long long *)a.v[" << F_ICNT << "];\n";
  o << "  const int *__restrict__ kc = (const int *)a.v[" << F_KC << "];\n";
  for (int i = 0; i < nx; ++i) {
    if (d.col[d.xslot[i]].dtype == LMFAO_U8)
      o << "  const unsigned char *__restrict__ xc" << i << " = (const unsigned char *)a.v[" << F_X0 + i << "];\n";
    else
      o << "  const float *__restrict__ xc" << i << " = (const float *)a.v[" << F_X0 + i << "];\n";
  }
  std::map<int, int> outer_arg;  // outer view -> argument slot of its FP64 rows
  for (int b = 0; b < (d.nfam ? d.nob : 0); ++b) {
    const int ov = d.obit_outer[b];
    if (!outer_arg.count(ov)) {
      const int slot = F_OV0 + (int)outer_arg.size();
      outer_arg[ov] = slot;
      o << "  const double *__restrict__ ov" << ov << " = (const double *)a.v[" << slot << "];\n";
    }
  }
  o << "  extern __shared__ __align__(16) unsigned char smem[];\n";
  o << "  T *tab = (T *)(smem + " << L.off_tab << ");\n";
  o << "  int *tcode = (int *)(smem + " << L.off_code << ");\n";
  o << "  T *Pf = (T *)(smem + " << L.off_pf << ");\n";
  o << "  unsigned int *Pi = (unsigned int *)(smem + " << L.off_pi << ");\n";
  o << "  float *hf0 = (float *)(smem + " << L.off_h << ");\n";
  o << "  float *hf = hf0 + warp * " << d.hist_f + d.hist_i << ";\n";
  o << "  unsigned int *hi = (unsigned int *)(hf + " << d.hist_f << ");\n";
  o << "  T *b4f = (T *)(smem + " << L.off_b4f << ");\n";
  o << "  unsigned int *b4i = (unsigned int *)(smem + " << L.off_b4i << ");\n";
  // staging: planar inner rows (values, then codes as int bits in FP32), zeroed accumulators
  if (d.ni) {
    const int rsw = fp64 ? L.rs : 4 * L.nfull + L.tew;  // staged words per row
    o << "#pragma unroll 4\n";
    o << "  for (int i = tid; i < " << nkeys * rsw << "; i += " << block << ") {\n";
    o << "    const int k = i / " << rsw << ", c = i - k * " << rsw << ";\n";
    o << "    T t = (T)0;\n";
    o << "    if (c < " << nw << ") t = gtab[(long long)k * " << nw << " + c];\n";
    if (!fp64)
      o << "    else if (c < " << nw + d.ncode << ") t = __int_as_float(gcod[(long long)k * " << d.ncode << " + c - " << nw
        << "]);\n";
    if (fp64) {
      o << "    tab[(c / 2) * " << nkeys * 2 << " + k * 2 + c % 2] = t;\n  }\n";
    } else {
      o << "    if (c < " << 4 * L.nfull << ") tab[(c / 4) * " << nkeys * 4 << " + k * 4 + c % 4] = t;\n";
      o << "    else tab[" << (long long)L.nfull * nkeys * 4 << " + k * " << L.tew << " + c - " << 4 * L.nfull
        << "] = t;\n  }\n";
    }
    if (fp64 && d.ncode)
      o << "  for (int i = tid; i < " << nkeys * d.ncode << "; i += " << block << ") tcode[i] = gcod[i];\n";
  }
  if (d.smem_p)
    o << "  for (int i = tid; i < " << nkeys * d.n3f * ls << "; i += " << block << ") Pf[i] = (T)0;\n";
  if (L.pi_smem)
    o << "  for (int i = tid; i < " << nkeys * d.n3i * ls << "; i += " << block << ") Pi[i] = 0u;\n";
  o << "  for (int i = tid; i < " << (long long)(block / 32) * (d.hist_f + d.hist_i) << "; i += " << block
    << ") hf0[i] = 0.f;\n";
  o << "  for (int i = tid; i < " << d.b4_fcells << "; i += " << block << ") b4f[i] = (T)0;\n";
  o << "  for (int i = tid; i < " << d.b4_icells << "; i += " << block << ") b4i[i] = 0u;\n";
  o << "  if (tid == 0) ticket = 0u;\n";
  o << "  __syncthreads();\n";

  // ---------------------------------------------------------------- per tuple
  o << "  auto tuple = [&](const int k";
  for (int i = 0; i < nx; ++i) o << ", const float xr" << i;
  o << ", const unsigned int obits, T (&acc)[" << VX << "], unsigned int (&hri)[" << std::max(1, NRI)
    << "], const T wsT, const unsigned long long ws) {\n";
  std::vector<std::string> v(nw), code(d.ncode);
  if (d.ni) {
    static const char *c4[4] = {"x", "y", "z", "w"};
    if (!fp64) {
      for (int q = 0; q < L.nfull; ++q)
        o << "    const float4 t" << q << " = reinterpret_cast<const float4 *>(tab)[" << (long long)q * nkeys
          << " + k];\n";
      const char *tt = L.tew == 4 ? "float4" : L.tew == 2 ? "float2" : "float";
      if (L.tew)
        o << "    const " << tt << " tt = reinterpret_cast<const " << tt << " *>(tab + " << (long long)L.nfull * nkeys * 4
          << ")[k];\n";
      auto word = [&](int p) {
        if (p < 4 * L.nfull) return "t" + std::to_string(p / 4) + "." + c4[p % 4];
        return L.tew == 1 ? std::string("tt") : "tt." + std::string(c4[p - 4 * L.nfull]);
      };
      for (int w = 0; w < nw; ++w) v[w] = word(w);
      for (int c = 0; c < d.ncode; ++c) code[c] = "__float_as_int(" + word(nw + c) + ")";
    } else {
      for (int q = 0; q < L.rs / 2; ++q)
        o << "    const double2 t" << q << " = reinterpret_cast<const double2 *>(tab)[" << (long long)q * nkeys
          << " + k];\n";
      for (int w = 0; w < nw; ++w) v[w] = "t" + std::to_string(w / 2) + (w % 2 ? ".y" : ".x");
      for (int c = 0; c < d.ncode; ++c)
        code[c] = "tcode[k * " + std::to_string(d.ncode) + " + " + std::to_string(c) + "]";
    }
    o << "    if (" << v[0] << " == (T)0) return;  // no partner in the inner relation\n";
  } else {
    v[0] = "(T)1";
  }
  for (int i = 0; i < nx; ++i) o << "    const T x" << i << " = (T)xr" << i << ";\n";
  // monomials
  for (int j = 0; j < nm; ++j) {
    std::string e;
    for (int i = 0; i < nx; ++i)
      for (int p = 0; p < d.mexp[j][i]; ++p) e += (e.empty() ? "" : " * ") + std::string("x") + std::to_string(i);
    o << "    T u" << j << " = " << (e.empty() ? "(T)1" : e) << ";\n";
  }
  for (int f = 0; f < d.nind; ++f) {
    const DFac &fc = d.ind[f];
    o << "    if (!(xr" << xidx(fc.col) << " " << cmp_src(fc.op) << " " << flt(fc.t) << ")) u" << d.ind_mono[f]
      << " = (T)0;\n";
  }
  for (int j = 0; j < nm; ++j)
    for (int w = 0; w < nw; ++w) o << "    acc[" << j * nw + w << "] += u" << j << " * " << v[w] << ";\n";
  // leaf of the tuple's filter (filters are disjoint)
  o << "    int leaf = -1;\n";
  if (d.nfam) {
    o << "    unsigned int bits = obits;\n";
    if (d.ibit_code >= 0) o << "    bits |= (unsigned int)" << code[d.ibit_code] << ";\n";
    for (int q = 0; q < d.nrb; ++q)
      o << "    if (xr" << xidx(d.rb[q].col) << " " << cmp_src(d.rb[q].op) << " " << flt(d.rb[q].t) << ") bits |= "
        << (1u << d.rb_pos[q]) << "u;\n";
    for (int f = 0; f < d.nfam; ++f)
      o << "    " << (f ? "else " : "") << "if ((bits & " << d.fmask[f] << "u) == " << d.fmask[f] << "u) leaf = " << f
        << ";\n";
  }
  // bucket codes of root columns, once per (column, thresholds)
  std::map<std::pair<int, std::pair<int, int>>, std::string> rcode;
  auto declare_rowcode = [&](const DGroupRef &q) {
    auto key = std::make_pair(xidx(q.a), std::make_pair(q.thr0, q.nthr));
    if (rcode.count(key)) return;
    const std::string name = "rc" + std::to_string(rcode.size());
    o << "    const int " << name << " = 0";
    for (int t = 0; t < q.nthr; ++t) o << " + (" << flt(thr[q.thr0 + t]) << " < xr" << key.first << ")";
    o << ";\n";
    rcode[key] = name;
  };
  for (int s = 0; s < d.nb1; ++s)
    for (int i = 0; i < d.b1[s].nref; ++i)
      if (d.b1[s].ref[i].src == 2) declare_rowcode(d.b1[s].ref[i]);
  for (const DGroupRef &q : grefs4)
    if (q.src == 2) declare_rowcode(q);
  auto rowcode = [&](const DGroupRef &q) -> std::string {
    return rcode.at(std::make_pair(xidx(q.a), std::make_pair(q.thr0, q.nthr)));
  };
  auto code_of = [&](const DGroupRef &q) -> std::string {
    if (q.src == 3) return code[q.b];
    if (q.src == 4) return "leaf";
    return rowcode(q);
  };
  auto sel_u = [&](int j) { return "u" + std::to_string(j); };
  // histogram sets
  for (int s = 0; s < d.nb1; ++s) {
    const DFastB1 &b = d.b1[s];
    o << "    {\n      int g = 0;\n      bool ok = true;\n";
    for (int i = 0; i < b.nref; ++i) {
      o << "      { const int c = " << code_of(b.ref[i]) << "; if (c < 0) ok = false; g += c * " << b.ref[i].stride
        << "; }\n";
    }
    o << "      if (ok) {\n";
    if (hoff[s] >= 0) {
      for (int c = 0; c < b.nf; ++c) o << "        const T vf" << c << " = " << sel_u(b.fj[c]) << " * " << v[b.fw[c]] << ";\n";
      for (int c = 0; c < b.ni; ++c)
        o << "        const unsigned int vi" << c << " = (unsigned int)(" << sel_u(b.ij[c]) << " * " << v[b.iw[c]] << ");\n";
      for (int gg = 0; gg < b.G; ++gg) {
        o << "        if (g == " << gg << ") {";
        for (int c = 0; c < b.nf; ++c) o << " acc[" << hoff[s] + gg * b.nf + c << "] += vf" << c << ";";
        for (int c = 0; c < b.ni; ++c) o << " hri[" << hoffi[s] + gg * b.ni + c << "] += vi" << c << ";";
        o << " }\n";
      }
    } else {
      for (int c = 0; c < b.nf; ++c)
        o << "        { const T val = " << sel_u(b.fj[c]) << " * " << v[b.fw[c]] << "; if (val != (T)0) atomicAdd(hf + "
          << b.smem_f << " + g * " << b.nf << " + " << c << ", (float)val); }\n";
      for (int c = 0; c < b.ni; ++c)
        o << "        { const T val = " << sel_u(b.ij[c]) << " * " << v[b.iw[c]] << "; if (val != (T)0) atomicAdd(hi + "
          << b.smem_i << " + g * " << b.ni << " + " << c << ", (unsigned int)val); }\n";
    }
    o << "      }\n    }\n";
  }
  // root-to-inner partials (split by leaf)
  if (d.n3) {
    o << "    if (" << (ls > 1 ? "leaf >= 0" : "true") << ") {\n";
    for (int c = 0; c < d.n3; ++c) {
      const std::string pc = std::to_string(d.p3col[c] * ls) + (ls > 1 ? " + leaf" : "");
      o << "      { const T val = " << sel_u(d.j3[c]) << "; if (val != (T)0) {";
      if (d.int3[c]) {
        o << " const unsigned long long iv = (unsigned long long)val * ws;";
        if (L.pi_smem) o << " atomicAdd(Pi + (long long)k * " << d.n3i * ls << " + " << pc << ", (unsigned int)iv);";
        else o << " atomicAdd(p3i + (long long)k * " << d.n3i * ls << " + " << pc << ", iv);";
      } else {
        if (d.smem_p) o << " atomicAdd(Pf + (long long)k * " << d.n3f * ls << " + " << pc << ", val * wsT);";
        else if (fp64) o << " atomicAdd(p3f + (long long)k * " << d.n3f * ls << " + " << pc << ", (double)(val * wsT));";
        else o << " atomicAdd(p3f32 + (long long)k * " << d.n3f * ls << " + " << pc << ", (float)(val * wsT));";
      }
      o << " } }\n";
    }
    o << "    }\n";
  }
  // CTA-private items: those of every filter, then those of the tuple's filter
  auto b4_item = [&](int i, const std::string &off) {
    o << "      { const T val = " << sel_u(d.b4_j[i]) << " * " << v[d.b4_w[i]] << ";\n";
    o << "        if (val != (T)0) {\n          long long cell = 0;\n          bool ok = true;\n";
    for (int gi = d.b4_g0[i]; gi < d.b4_g0[i] + d.b4_ng[i]; ++gi) {
      const DGroupRef &q = grefs4[gi];
      o << "          { const int c = " << code_of(q) << "; if (c < 0) ok = false; cell += (long long)c * " << q.stride
        << "; }\n";
    }
    o << "          if (ok) ";
    if (d.b4_int[i])
      o << "atomicAdd(b4i + " << d.b4_so[i] << off << " + cell * " << d.b4_cellmul[i]
        << ", (unsigned int)val * (unsigned int)ws);\n";
    else
      o << "atomicAdd(b4f + " << d.b4_so[i] << off << " + cell * " << d.b4_cellmul[i] << ", val * wsT);\n";
    o << "        }\n      }\n";
  };
  if (d.nb4) {
    o << "    {\n";
    for (int i = d.b4_off[0]; i < d.b4_off[1]; ++i) b4_item(i, "");
    o << "    }\n";
    // Filters whose items differ only by a constant shift of their output cells per filter
    // index (the leaves of a decision-tree level ask the same questions) run one copy of the
    // items with the tuple's filter index in the address: no divergence over the filters.
    const int n0 = d.nfam ? d.b4_off[2] - d.b4_off[1] : 0;
    bool uniform = d.nfam > 1 && n0 > 0;
    long long dint = 0, dflt = 0;  // per-filter shift of the integral / float cells
    bool hint = false, hflt = false;
    for (int f = 1; f < d.nfam && uniform; ++f) {
      if (d.b4_off[f + 2] - d.b4_off[f + 1] != n0) { uniform = false; break; }
      for (int k = 0; k < n0 && uniform; ++k) {
        const int a = d.b4_off[1] + k, b = d.b4_off[f + 1] + k;
        if (d.b4_j[a] != d.b4_j[b] || d.b4_w[a] != d.b4_w[b] || d.b4_int[a] != d.b4_int[b] ||
            d.b4_ng[a] != d.b4_ng[b] || d.b4_cellmul[a] != d.b4_cellmul[b]) {
          uniform = false;
          break;
        }
        for (int g = 0; g < d.b4_ng[a] && uniform; ++g) {
          const DGroupRef &qa = grefs4[d.b4_g0[a] + g], &qb = grefs4[d.b4_g0[b] + g];
          if (qa.src != qb.src || qa.a != qb.a || qa.b != qb.b || qa.kind != qb.kind || qa.thr0 != qb.thr0 ||
              qa.nthr != qb.nthr || qa.stride != qb.stride)
            uniform = false;
        }
        long long &dl = d.b4_int[a] ? dint : dflt;
        bool &has = d.b4_int[a] ? hint : hflt;
        const long long sh = (long long)(d.b4_so[b] - d.b4_so[a]);
        if (sh % f) uniform = false;
        else if (!has) { dl = sh / f; has = true; }
        else if (dl != sh / f) uniform = false;
      }
    }
    if (uniform) {
      o << "    if (leaf >= 0) {\n";
      o << "      const int lo_i = leaf * " << dint << ", lo_f = leaf * " << dflt << ";\n";
      for (int k = 0; k < n0; ++k) {
        const int i = d.b4_off[1] + k;
        b4_item(i, d.b4_int[i] ? " + lo_i" : " + lo_f");
      }
      o << "    }\n";
    } else if (d.nfam) {
      o << "    switch (leaf) {\n";
      for (int f = 0; f < d.nfam; ++f) {
        if (d.b4_off[f + 2] <= d.b4_off[f + 1]) continue;
        o << "    case " << f << ": {\n";
        for (int i = d.b4_off[f + 1]; i < d.b4_off[f + 2]; ++i) b4_item(i, "");
        o << "      break;\n    }\n";
      }
      o << "    default: break;\n    }\n";
    }
  }
  o << "  };\n\n";

  // ---------------------------------------------------------------- work items
  auto xreg_type = [&](int i) {
    return d.col[d.xslot[i]].dtype == LMFAO_U8 ? std::string("unsigned int") : std::string("float4");
  };
  auto xreg_load = [&](int i, const std::string &q) {
    if (d.col[d.xslot[i]].dtype == LMFAO_U8)
      return "reinterpret_cast<const unsigned int *>(xc" + std::to_string(i) + ")[" + q + "]";
    return "reinterpret_cast<const float4 *>(xc" + std::to_string(i) + ")[" + q + "]";
  };
  auto xcomp = [&](int i, const std::string &reg, int u) {
    static const char *c4[4] = {"x", "y", "z", "w"};
    if (d.col[d.xslot[i]].dtype == LMFAO_U8) return "(float)((" + reg + " >> " + std::to_string(8 * u) + ") & 0xffu)";
    return reg + "." + c4[u];
  };
  auto quad_load = [&](const std::string &q, const std::string &ind) {
    if (d.ni) o << ind << "kn = reinterpret_cast<const int4 *>(kc)[" << q << "];\n";
    for (int i = 0; i < nx; ++i) o << ind << "xn" << i << " = " << xreg_load(i, q) << ";\n";
  };
  o << "  int wi;\n";
  o << "  {\n    unsigned int t = 0u;\n    if (lane == 0) t = atomicAdd(&ticket, 1u);\n";
  o << "    wi = ib + (int)__shfl_sync(0xffffffffu, t, 0);\n  }\n";
  o << "  Work wk = {0, 0, 0};\n  unsigned long long ws = 0ull;\n";
  o << "  if (wi < nwork) { wk = work[wi]; ws = wseg[wk.seg]; }\n";
  o << "  long long qa = (wk.r0 + 3) >> 2, qe = (wk.r0 + wk.len) >> 2;\n";
  o << "  if (qe < qa) qe = qa;\n";
  if (d.ni) o << "  int4 kn = make_int4(0, 0, 0, 0);\n";
  for (int i = 0; i < nx; ++i) o << "  " << xreg_type(i) << " xn" << i << "{};\n";
  o << "  long long q = qa + lane;\n  if (q < qe) {\n";
  quad_load("q", "    ");
  o << "  }\n";
  o << "  while (wi < nwork) {\n";
  o << "    int wn;  // the next item (shared-memory ticket): its record is requested now\n";
  o << "    {\n      unsigned int t = 0u;\n      if (lane == 0) t = atomicAdd(&ticket, 1u);\n";
  o << "      wn = ib + (int)__shfl_sync(0xffffffffu, t, 0);\n    }\n";
  o << "    Work wkn = {0, 0, 0};\n";
  o << "    if (wn < nwork) wkn = work[wn];  // used after the tuples of this item\n";
  o << "    const T wsT = (T)ws;\n";
  o << "    T acc[" << VX << "];\n";
  o << "#pragma unroll\n    for (int i = 0; i < " << VX << "; ++i) acc[i] = (T)0;\n";
  o << "    unsigned int hri[" << std::max(1, NRI) << "];\n";
  o << "#pragma unroll\n    for (int i = 0; i < " << std::max(1, NRI) << "; ++i) hri[i] = 0u;\n";
  o << "    if (ws != 0ull) {\n";
  // outer predicate bits of the segment
  o << "      unsigned int obits = 0u;\n";
  if (d.nfam && d.nob) {
    o << "      {\n        unsigned int mine = 0u;\n        const long long sg = wk.seg;\n";
    for (int b = 0; b < d.nob; ++b) {
      const DOuter &ov = d.outer[d.obit_outer[b]];
      o << "        if (lane == " << b << ") {\n          long long ok = 0;\n";
      for (int i = 0; i < d.seg.ndig; ++i)
        if (ov.dstride[i])
          o << "          ok += ((sg / " << d.seg.radix[i] << "ll) % " << d.seg.dom[i] << "ll) * " << ov.dstride[i]
            << "ll;\n";
      o << "          if (ov" << d.obit_outer[b] << "[ok * " << ov.v.ncols << " + " << d.obit_col[b]
        << "] > 0.0) mine = " << (1u << d.obit_pos[b]) << "u;\n        }\n";
    }
    o << "        obits = __reduce_or_sync(0xffffffffu, mine);\n      }\n";
  }
  o << "      const long long r0 = wk.r0, rend = r0 + wk.len;\n";
  o << "      const long long he = 4 * qa < rend ? 4 * qa : rend;\n";
  o << "      const long long te = 4 * qe > he ? 4 * qe : he;\n";
  o << "      {\n        long long r = -1;\n";
  o << "        if (lane < 4) { if (r0 + lane < he) r = r0 + lane; }\n";
  o << "        else if (lane >= 8 && lane < 12) { if (te + (lane - 8) < rend) r = te + (lane - 8); }\n";
  o << "        if (r >= 0) tuple(" << (d.ni ? "kc[r]" : "0");
  for (int i = 0; i < nx; ++i) o << ", (float)xc" << i << "[r]";
  o << ", obits, acc, hri, wsT, ws);\n      }\n";
  o << "      for (; q < qe; q += 32) {\n";
  if (d.ni) o << "        const int4 kk = kn;\n";
  for (int i = 0; i < nx; ++i) o << "        const " << xreg_type(i) << " xk" << i << " = xn" << i << ";\n";
  o << "        if (q + 32 < qe) {\n";
  quad_load("q + 32", "          ");
  o << "        }\n";
  static const char *comp[4] = {"x", "y", "z", "w"};
  for (int u = 0; u < 4; ++u) {
    o << "        tuple(" << (d.ni ? std::string("kk.") + comp[u] : std::string("0"));
    for (int i = 0; i < nx; ++i) o << ", " << xcomp(i, "xk" + std::to_string(i), u);
    o << ", obits, acc, hri, wsT, ws);\n";
  }
  o << "      }\n    }\n";
  o << "    unsigned long long wsn = 0ull;\n";
  o << "    if (wn < nwork) wsn = wseg[wkn.seg];\n";
  o << "    long long qan = (wkn.r0 + 3) >> 2, qen = (wkn.r0 + wkn.len) >> 2;\n";
  o << "    if (qen < qan) qen = qan;\n";
  o << "    q = qan + lane;\n    if (q < qen) {\n";
  quad_load("q", "      ");
  o << "    }\n";
  o << "    if (ws != 0ull) {\n";
  // per-segment sums: reduce-scatter over the warp
  const WarpReduce wr = gen_warp_reduce(VX, "      ");
  o << wr.src;
  if (VX == V) {
    o << gen_reduce_flush(wr, "phi0f", "(long long)wk.seg * " + std::to_string(V), "      ");
  } else {  // the segment sums, then the float cells of the register histograms
    const int mask = (1 << wr.shift) - 1;
    o << "      { const int i = lane >> " << wr.shift << ";\n";
    o << "        if (" << (mask ? "(lane & " + std::to_string(mask) + ") == 0 && " : "") << "r_[0] != (T)0) {\n";
    o << "          if (i < " << V << ") atomicAdd(phi0f + (long long)wk.seg * " << V << " + i, r_[0]);\n";
    for (int s = 0; s < d.nb1; ++s) {
      const DFastB1 &b = d.b1[s];
      if (hoff[s] < 0 || !b.nf) continue;
      o << "          else if (i >= " << hoff[s] << " && i < " << hoff[s] + b.G * b.nf << ") atomicAdd(phi1f + (long long)wk.seg * "
        << d.phi1f_seg << " + " << b.gbase_f << " + (i - " << hoff[s] << "), (float)r_[0]);\n";
    }
    o << "        }\n      }\n";
  }
  for (int s = 0; s < d.nb1; ++s) {  // the integral cells of the register histograms
    const DFastB1 &b = d.b1[s];
    for (int k = 0; hoffi[s] >= 0 && k < b.G * b.ni; ++k)
      o << "      { const unsigned int x = __reduce_add_sync(0xffffffffu, hri[" << hoffi[s] + k
        << "]); if (lane == 0 && x) atomicAdd(phi1i + (long long)wk.seg * " << d.phi1i_seg << " + " << b.gbase_i << " + "
        << k << ", x); }\n";
  }
  if (d.n0i) {
    o << "      {\n        T iv = (T)0;\n";
    for (int e = 0; e < d.n0i; ++e) {
      const int qq = d.i0j[e] * nw + d.i0w[e];
      o << "        { const T t = __shfl_sync(0xffffffffu, r_[" << wr.reg_of(qq) << "], " << wr.lane_of(qq)
        << "); if (lane == " << e << ") iv = t; }\n";
    }
    o << "        if (lane < " << d.n0i << ") {\n";
    o << "          const unsigned long long it = (unsigned long long)(iv + (T)0.5);\n";
    o << "          if (it) atomicAdd(phi0i + (long long)wk.seg * " << d.n0i << " + lane, it);\n        }\n      }\n";
  }
  if (d.nb1) {
    o << "      __syncwarp();\n";
    for (int s = 0; s < d.nb1; ++s) {
      const DFastB1 &b = d.b1[s];
      if (hoff[s] >= 0) continue;  // in registers
      if (b.nf)
        o << "      for (int i = lane; i < " << (long long)b.G * b.nf << "; i += 32) { const float x = hf[" << b.smem_f
          << " + i]; if (x != 0.f) { hf[" << b.smem_f << " + i] = 0.f; atomicAdd(phi1f + (long long)wk.seg * "
          << d.phi1f_seg << " + " << b.gbase_f << " + i, x); } }\n";
      if (b.ni)
        o << "      for (int i = lane; i < " << (long long)b.G * b.ni << "; i += 32) { const unsigned int x = hi["
          << b.smem_i << " + i]; if (x) { hi[" << b.smem_i << " + i] = 0u; atomicAdd(phi1i + (long long)wk.seg * "
          << d.phi1i_seg << " + " << b.gbase_i << " + i, x); } }\n";
    }
    o << "      __syncwarp();\n";
  }
  o << "    }\n";
  o << "    wi = wn;\n    wk = wkn;\n    ws = wsn;\n    qa = qan;\n    qe = qen;\n";
  o << "  }\n";
  // end of the CTA: shared partials and CTA-private items to the outputs
  o << "  __syncthreads();\n";
  if (d.smem_p)
    o << "  for (int i = tid; i < " << nkeys * d.n3f * ls << "; i += " << block
      << ") if (Pf[i] != (T)0) atomicAdd(p3f + i, (double)Pf[i]);\n";
  if (L.pi_smem)
    o << "  for (int i = tid; i < " << nkeys * d.n3i * ls << "; i += " << block
      << ") if (Pi[i]) atomicAdd(p3i + i, (unsigned long long)Pi[i]);\n";
  for (const DMirror &mr : mirror) {
    if (mr.integral)
      o << "  for (int i = tid; i < " << mr.len << "; i += " << block << ") if (b4i[" << mr.soff
        << " + i]) atomicAdd(icnt + " << mr.gout << "ll + i, (unsigned long long)b4i[" << mr.soff << " + i]);\n";
    else
      o << "  for (int i = tid; i < " << mr.len << "; i += " << block << ") if (b4f[" << mr.soff
        << " + i] != (T)0) atomicAdd(fsum + " << mr.gout << "ll + i, (double)b4f[" << mr.soff << " + i]);\n";
  }
  o << "}\n";
  return o.str();
}

}  // namespace lmfao
