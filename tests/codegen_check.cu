// Test program: builds the sources that the plan-time code generators write for a few
// representative shapes and compiles them with NVRTC for sm_103a (no GPU needed). Prints one
// line per shape: "<name> ok <registers> <spill bytes>" or "<name> FAIL <log>".
#include <nvrtc.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../paper_2008_08657_b300/csrc/codegen.h"

using namespace lmfao;

static void check(const char *name, const std::string &src) {
  nvrtcProgram prog;
  nvrtcCreateProgram(&prog, src.c_str(), "gen.cu", 0, nullptr, nullptr);
  const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--ptxas-options=-v"};
  const nvrtcResult r = nvrtcCompileProgram(prog, 3, opts);
  size_t n = 0;
  nvrtcGetProgramLogSize(prog, &n);
  std::string log(n, '\0');
  if (n) nvrtcGetProgramLog(prog, &log[0]);
  nvrtcDestroyProgram(&prog);
  if (r != NVRTC_SUCCESS) {
    printf("%s FAIL %s\n", name, log.substr(0, 300).c_str());
    return;
  }
  int regs = -1, spill = -1;
  size_t p = log.find("Used ");
  if (p != std::string::npos) sscanf(log.c_str() + p, "Used %d registers", &regs);
  p = log.find("bytes spill stores");
  if (p != std::string::npos) {
    size_t q = log.rfind(',', p);
    if (q != std::string::npos) sscanf(log.c_str() + q + 1, "%d", &spill);
  }
  printf("%s ok %d %d\n", name, regs, spill);
}

static DFast lean_base() {
  DFast d{};
  d.lean = 1; d.vec = 1; d.smem_view = 1; d.smem_p = 1; d.nk = 1;
  d.col[0] = DCol{nullptr, LMFAO_I32}; d.col[1] = DCol{nullptr, LMFAO_F32}; d.col[2] = DCol{nullptr, LMFAO_U8};
  d.kslot[0] = 0;
  return d;
}

// A Weather-like view (2 key columns, 8 float attributes; columns 1, w_i, w_i w_j) and an
// Item-like one (a categorical code, a bucketed code, an indicator factor).
static void check_views() {
  static int dummy_keyrow = 0;
  DViewKernel d{};
  d.keyrow = &dummy_keyrow;
  d.nkeys = 161200;
  d.ncolsin = 10;
  for (int i = 0; i < 10; ++i) d.in[i] = DCol{nullptr, i < 2 ? LMFAO_I32 : LMFAO_F32};
  std::vector<int> cfo{0};
  std::vector<DFac> facs;
  cfo.push_back(0);  // COUNT
  for (int a = 0; a < 8; ++a) { facs.push_back(DFac{2 + a, 0, 1, 0, 0.f}); cfo.push_back((int)facs.size()); }
  for (int a = 0; a < 8; ++a)
    for (int b = a; b < 8; ++b) {
      if (a == b) facs.push_back(DFac{2 + a, 0, 2, 0, 0.f});
      else { facs.push_back(DFac{2 + a, 0, 1, 0, 0.f}); facs.push_back(DFac{2 + b, 0, 1, 0, 0.f}); }
      cfo.push_back((int)facs.size());
    }
  d.ncols = (int)cfo.size() - 1;
  std::vector<int4> cdesc;
  std::vector<float> thr;
  check("view_weather", gen_view_source(d, cfo, facs, cdesc, thr));
  DViewKernel e{};
  e.keyrow = &dummy_keyrow;
  e.nkeys = 3700;
  e.ncolsin = 4;
  e.in[0] = DCol{nullptr, LMFAO_I32}; e.in[1] = DCol{nullptr, LMFAO_F32}; e.in[2] = DCol{nullptr, LMFAO_I32};
  e.in[3] = DCol{nullptr, LMFAO_U8};
  std::vector<int> cfo2{0, 0, 1, 3};
  std::vector<DFac> facs2{DFac{1, 0, 1, 0, 0.f}, DFac{1, 0, 2, 0, 0.f}, DFac{3, 1, 1, LMFAO_GT, 0.5f}};
  e.ncols = 3;
  std::vector<int4> cdesc2{make_int4(2, 0, 0, 0), make_int4(1, LMFAO_GB_BUCKET, 0, 3)};
  std::vector<float> thr2{-1.f, 0.f, 1.f};
  e.ncodes = 2;
  check("view_item", gen_view_source(e, cfo2, facs2, cdesc2, thr2));
}

int main() {
  check_views();
  for (int fp64 = 0; fp64 < 2; ++fp64) {
    const int block = fp64 ? 512 : 1024;
    const std::string sfx = fp64 ? "_fp64" : "_fp32";
    {  // Retailer-like lean pass: one value column, five inner columns, one histogram set
      DFast d = lean_base();
      d.ni = 1; d.nx = 1; d.xslot[0] = 1; d.nw = 5; d.nm = 3; d.nkeys = 3700; d.ncode = 1;
      d.nb1 = 1; d.b1[0].G = 50; d.b1code[0] = 0; d.hist_i = 50; d.phi1i_seg = 50;
      d.n3 = 2; d.j3[0] = 0; d.int3[0] = 1; d.p3col[0] = 0; d.j3[1] = 1; d.p3col[1] = 0; d.n3f = 1; d.n3i = 1;
      d.n0i = 1;
      check(("lean_retailer" + sfx).c_str(), gen_root_pass_source(d, fp64, block));
      d.lanes = 1;
      check(("lean_retailer_lanes" + sfx).c_str(), gen_root_pass_source(d, fp64, block));
    }
    {  // Favorita-like lean pass: a float and a uint8 value column, three histogram sets
      DFast d = lean_base();
      d.ni = 1; d.nx = 2; d.xslot[0] = 1; d.xslot[1] = 2; d.nw = 1; d.nm = 6; d.nkeys = 4100; d.ncode = 3;
      d.nb1 = 3;
      const int G[3] = {33, 337, 2};
      int off = 0;
      for (int b = 0; b < 3; ++b) { d.b1[b].G = G[b]; d.b1[b].smem_i = off; d.b1[b].gbase_i = off; d.b1code[b] = b; off += G[b]; }
      d.hist_i = off; d.phi1i_seg = off;
      d.n3 = 3; d.int3[0] = 1; d.j3[1] = 1; d.j3[2] = 2; d.p3col[2] = 1; d.n3f = 2; d.n3i = 1;
      check(("lean_favorita" + sfx).c_str(), gen_root_pass_source(d, fp64, block));
    }
    {  // no inner relation, three value columns
      DFast d = lean_base();
      d.ni = 0; d.nx = 3; d.xslot[0] = 1; d.xslot[1] = 1; d.xslot[2] = 2; d.nw = 1; d.nm = 10; d.n0i = 1;
      check(("lean_no_inner" + sfx).c_str(), gen_root_pass_source(d, fp64, block));
    }
    {  // decision-tree level: 8 leaves from outer, inner and root predicate bits; leaf histograms,
       // leaf-split partials and per-leaf CTA-private bucket items
      DFast d = lean_base();
      d.lean = 0; d.smem_p = 0;
      d.ni = 1; d.nx = 1; d.xslot[0] = 1; d.nw = 1; d.nm = 3; d.nkeys = 3700; d.ncode = 2;
      d.mexp[1][0] = 1; d.mexp[2][0] = 2;
      d.nb1 = 1; d.b1[0].nref = 2;
      d.b1[0].ref[0] = DGroupRef{3, 0, 0, 0, 0, 0, 8};
      d.b1[0].ref[1] = DGroupRef{4, 0, 0, 0, 0, 0, 1};
      d.b1[0].G = 20; d.b1[0].nf = 2; d.b1[0].fj[0] = 1; d.b1[0].fj[1] = 2; d.b1[0].ni = 1;
      d.hist_f = 40; d.hist_i = 20; d.phi1f_seg = 40; d.phi1i_seg = 20;
      d.n3 = 3; d.int3[0] = 1; d.j3[1] = 1; d.j3[2] = 2; d.p3col[2] = 1; d.n3f = 2; d.n3i = 1; d.b3leaf = 8;
      d.n0i = 1;
      d.nfam = 8;
      for (int f = 0; f < 8; ++f) d.fmask[f] = (unsigned)f | 8u;
      d.nob = 2; d.obit_outer[1] = 1; d.obit_col[0] = 1; d.obit_col[1] = 2; d.obit_pos[1] = 1;
      d.ibit_code = 1; d.nrb = 1; d.rb[0] = DFac{1, 1, 1, LMFAO_LE, 0.5f}; d.rb_pos[0] = 2;
      d.nouter = 2; d.outer[0].v.ncols = 10; d.outer[0].dstride[0] = 124; d.outer[0].dstride[1] = 1;
      d.outer[1].v.ncols = 5; d.outer[1].dstride[0] = 1;
      d.seg.ndig = 2; d.seg.dom[0] = 1300; d.seg.dom[1] = 124; d.seg.radix[0] = 124; d.seg.radix[1] = 1;
      d.nb4 = 24;
      for (int f = 0; f < 8; ++f) d.b4_off[f + 2] = 3 * (f + 1);
      std::vector<DGroupRef> g4;
      for (int i = 0; i < 24; ++i) {
        d.b4_j[i] = i % 3; d.b4_int[i] = i % 3 == 0; d.b4_g0[i] = i; d.b4_ng[i] = 1; d.b4_so[i] = (i / 3) * 20;
        d.b4_cellmul[i] = 3;
        g4.push_back(DGroupRef{2, 1, 0, LMFAO_GB_BUCKET, 0, 19, 1});
      }
      d.b4_fcells = 200; d.b4_icells = 200;
      std::vector<DMirror> mir{DMirror{1000, 0, 160, 0, 0}, DMirror{5000, 0, 160, 1, 0}};
      std::vector<float> thr(19);
      for (int i = 0; i < 19; ++i) thr[i] = 0.1f * i;
      std::string why;
      if (!family_eligible(d, why, g4)) printf("dt_level%s FAIL not eligible: %s\n", sfx.c_str(), why.c_str());
      else check(("dt_level" + sfx).c_str(), gen_family_source(d, fp64, block, thr, g4, mir));
      // the per-segment sums by leaf alone (8 cells of 2 float and 1 integral column): kept in
      // registers and reduced over the warp with the segment sums
      d.b1[0].nref = 1;
      d.b1[0].ref[0] = DGroupRef{4, 0, 0, 0, 0, 0, 1};
      d.b1[0].G = 8;
      d.hist_f = 16; d.hist_i = 8; d.phi1f_seg = 16; d.phi1i_seg = 8;
      if (!family_eligible(d, why, g4)) printf("dt_leaf_sums%s FAIL not eligible: %s\n", sfx.c_str(), why.c_str());
      else check(("dt_leaf_sums" + sfx).c_str(), gen_family_source(d, fp64, block, thr, g4, mir));
    }
    {  // general pass without an inner relation: two value columns (float and uint8), an
       // indicator factor and CTA-private items grouped by buckets of both columns
      DFast d = lean_base();
      d.lean = 0; d.smem_p = 0;
      d.ni = 0; d.nx = 2; d.xslot[0] = 1; d.xslot[1] = 2; d.nw = 1; d.nm = 4;
      d.mexp[1][0] = 1; d.mexp[2][1] = 1; d.mexp[3][0] = 2;
      d.nind = 1; d.ind[0] = DFac{1, 1, 1, LMFAO_GT, 0.25f}; d.ind_mono[0] = 2;
      d.nb4 = 2; d.b4_off[0] = 0; d.b4_off[1] = 2;
      std::vector<DGroupRef> g4{DGroupRef{2, 1, 0, LMFAO_GB_BUCKET, 3, 4, 1}, DGroupRef{2, 2, 0, LMFAO_GB_BUCKET, 0, 3, 1}};
      d.b4_j[0] = 0; d.b4_int[0] = 1; d.b4_g0[0] = 0; d.b4_ng[0] = 1; d.b4_so[0] = 0; d.b4_cellmul[0] = 1;
      d.b4_j[1] = 3; d.b4_g0[1] = 1; d.b4_ng[1] = 1; d.b4_so[1] = 0; d.b4_cellmul[1] = 1;
      d.b4_fcells = 8; d.b4_icells = 8;
      std::vector<DMirror> mir{DMirror{0, 0, 8, 1, 0}, DMirror{0, 0, 8, 0, 0}};
      std::vector<float> thr{0.5f, 1.5f, 2.5f, -1.f, 0.f, 1.f, 2.f};
      std::string why;
      if (!family_eligible(d, why, g4)) printf("general_no_inner%s FAIL not eligible: %s\n", sfx.c_str(), why.c_str());
      else check(("general_no_inner" + sfx).c_str(), gen_family_source(d, fp64, block, thr, g4, mir));
    }
  }
  return 0;
}
