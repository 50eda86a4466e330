// Host runs of the colour-split kernels beside their plain-layout counterparts (their
// text extracted from the sources; see tests/test_split_host.py). The launch is a loop
// over every block and thread. Modes:
//   split n B in.bin perm.bin out.bin            (FP32 nodal-coefficient kernels)
//     in.bin   float32: kn, g, u (B n^3 each, plain layout), k0 (float64, B n^3), ec
//              (float32, B nc^3, plain), r (float32, B n^3, plain)
//     perm.bin int64: for every plain index of B n^3 (then of B nc^3), its index in the
//              colour-split storage (computed by the test from the definition)
//     out.bin  float32: u after a red and a black pass (plain kernel, then split kernel
//              mapped back), r~ of the nodal residual (plain, split), u + P ec (plain,
//              split mapped back), 4 FW(r) (plain, split mapped back), 1/k (plain, split
//              mapped back)
//   split64 n B in.bin perm.bin out.bin          (FP64 stored-face kernels)
//     in.bin   float64: k0, g, u (B n^3 each, plain), ec (B nc^3), r (B n^3)
//     out.bin  float64, each plain then split mapped back: Kx, Ky, Kz, D, 1/D, u after a
//              red and a black pass, r~, then u + P ec of k_prolong against the block
//              form (plain; split mapped back; FP32 widened), FW(r) (B nc^3), u through
//              the plain -> split -> plain copies, u + P1 ec, the P1 restriction (B nc^3)
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

struct dim3 {
  unsigned x = 1, y = 1, z = 1;
  dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};
static dim3 blockIdx, threadIdx, blockDim, gridDim;
static float __fdividef(float a, float b) { return a / b; }
static float __fadd_rn(float a, float b) { return a + b; }
static float __fmul_rn(float a, float b) { return a * b; }
static float __fdiv_rn(float a, float b) { return a / b; }
static double __dadd_rn(double a, double b) { return a + b; }
static double __dmul_rn(double a, double b) { return a * b; }
static double __ddiv_rn(double a, double b) { return a / b; }
static float __double2float_rn(double a) { return (float)a; }
static double widen(float x) { return (double)x; }
// block-wide sums are compiled but never reached here (no partials are requested)
static double __shfl_down_sync(unsigned, double v, int) { return v; }
static void __syncthreads() {}
#define __shared__ static
using std::min;
static int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
struct float4 {
  float x, y, z, w;
};
static float4 make_float4(float a, float b, float c, float d) { return float4{a, b, c, d}; }
struct double2 {
  double x, y;
};
static double2 make_double2(double a, double b) { return double2{a, b}; }
static float fmaf_(float a, float b, float c) { return std::fmaf(a, b, c); }
#define fmaf fmaf_
using std::fma;

#include "split_kernels.inc"

template <typename F>
static void launch(dim3 grid, dim3 block, F body) {
  gridDim = grid;
  blockDim = block;
  for (unsigned bz = 0; bz < grid.z; ++bz)
    for (unsigned by = 0; by < grid.y; ++by)
      for (unsigned bx = 0; bx < grid.x; ++bx)
        for (unsigned t = 0; t < block.x; ++t) {
          blockIdx = dim3(bx, by, bz);
          threadIdx = dim3(t, 0, 0);
          body();
        }
}

template <typename T>
static std::vector<T> readv(FILE* f, size_t n) {
  std::vector<T> v(n);
  if (std::fread(v.data(), sizeof(T), n, f) != n) std::exit(3);
  return v;
}

static int split64(char** argv);

int main(int argc, char** argv) {
  if (argc < 7) return 2;
  if (std::string(argv[1]) == "split64") return split64(argv);
  if (std::string(argv[1]) != "split") return 2;
  const int n = std::atoi(argv[2]), B = std::atoi(argv[3]), nc = (n + 1) / 2;
  const size_t n3 = (size_t)n * n * n, nc3 = (size_t)nc * nc * nc;
  FILE* fi = std::fopen(argv[4], "rb");
  FILE* fp = std::fopen(argv[5], "rb");
  if (!fi || !fp) return 3;
  auto kn = readv<float>(fi, B * n3), g = readv<float>(fi, B * n3), u = readv<float>(fi, B * n3);
  auto k0 = readv<double>(fi, B * n3);
  auto ec = readv<float>(fi, B * nc3), r = readv<float>(fi, B * n3);
  auto perm = readv<int64_t>(fp, B * n3), permc = readv<int64_t>(fp, B * nc3);
  std::fclose(fi);
  std::fclose(fp);
  const float nan = std::numeric_limits<float>::quiet_NaN();
  const size_t ns = mlmc::split_elems(n), nsc = mlmc::split_elems(nc);
  auto to_split = [&](const std::vector<float>& a, const std::vector<int64_t>& pm, size_t total) {
    std::vector<float> b(total, nan);  // slots without a node stay NaN: reading one poisons the result
    for (size_t i = 0; i < a.size(); ++i) b[pm[i]] = a[i];
    return b;
  };
  auto from_split = [&](const std::vector<float>& b, const std::vector<int64_t>& pm) {
    std::vector<float> a(pm.size());
    for (size_t i = 0; i < pm.size(); ++i) a[i] = b[pm[i]];
    return a;
  };
  const unsigned T = 64;
  std::vector<float> out;
  // a red and a black pass
  std::vector<float> up = u, us = to_split(u, perm, B * ns), ks = to_split(kn, perm, B * ns),
                     gs = to_split(g, perm, B * ns);
  const int m = n - 2, half = (n - 1) / 2, P = mlmc::split_pitch(n);
  for (int c = 0; c < 2; ++c) {
    launch(dim3((unsigned)((m * half + T - 1) / T), (unsigned)(B * m)), dim3(T),
           [&] { mlmc::k_rbgs_nodal(c, n, B, kn.data(), g.data(), up.data(), nullptr); });
    MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)((m * (P / 4) + 127) / 128), (unsigned)m, (unsigned)B), dim3(128), [&] {
      mlmc::k_rbgs_split<LG>(c, ks.data(), gs.data(), us.data(), nullptr);
    }));
  }
  auto usb = from_split(us, perm);
  out.insert(out.end(), up.begin(), up.end());
  out.insert(out.end(), usb.begin(), usb.end());
  // the nodal residual of the swept iterate
  std::vector<float> rp(B * n3, nan), rss(B * ns, 0.0f);
  launch(dim3((unsigned)((n * n + T - 1) / T), (unsigned)(B * n)), dim3(T),
         [&] { mlmc::k_residual_nodal(n, B, kn.data(), g.data(), up.data(), rp.data(), nullptr); });
  MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)((m * (P / 4) + 127) / 128), (unsigned)(2 * m), (unsigned)B), dim3(128), [&] {
    mlmc::k_residual_split<LG>(ks.data(), gs.data(), us.data(), rss.data(), nullptr);
  }));
  auto rs = from_split(rss, perm);  // the split residual leaves boundary slots unwritten (zero here)
  out.insert(out.end(), rp.begin(), rp.end());
  out.insert(out.end(), rs.begin(), rs.end());
  // the trilinear correction
  std::vector<float> pp = u, ps = to_split(u, perm, B * ns), ecs = to_split(ec, permc, B * nsc);
  const int P2 = n - 1;
  launch(dim3((unsigned)((m * P2 + T - 1) / T), (unsigned)(B * m)), dim3(T),
         [&] { mlmc::k_prolong<float>(n, B, ec.data(), pp.data(), nullptr); });
  MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)((m * (P / 4) + 127) / 128), (unsigned)m, (unsigned)(2 * B)), dim3(128), [&] {
    mlmc::k_prolong_split<LG>(ecs.data(), ps.data(), nullptr);
  }));
  auto psb = from_split(ps, perm);
  out.insert(out.end(), pp.begin(), pp.end());
  out.insert(out.end(), psb.begin(), psb.end());
  // full weighting into the plain and the split coarse storage
  std::vector<float> gcp(B * nc3, 0.0f), gcs(B * nsc, 0.0f), r_s = to_split(r, perm, B * ns);
  const int hc = nc - 1;
  launch(dim3((unsigned)(((nc - 2) * hc + T - 1) / T), (unsigned)(B * (nc - 2))), dim3(T),
         [&] { mlmc::k_restrict<float, false>(n, B, r.data(), gcp.data(), nullptr); });
  MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)(((nc - 2) * (nc - 2) + 127) / 128), (unsigned)(nc - 2), (unsigned)B),
                                dim3(128), [&] { mlmc::k_restrict_split<LG>(r_s.data(), gcs.data(), nullptr); }));
  auto gcsb = from_split(gcs, permc);
  out.insert(out.end(), gcp.begin(), gcp.end());
  out.insert(out.end(), gcsb.begin(), gcsb.end());
  // the reciprocal nodal coefficient
  std::vector<float> knp(B * n3, nan), kns(B * ns, nan);
  launch(dim3((unsigned)((n * n + T - 1) / T), (unsigned)(B * n)), dim3(T),
         [&] { mlmc::k_nodal_k<float>(k0.data(), n, 1, n, B, knp.data()); });
  launch(dim3((unsigned)((n * n + T - 1) / T), (unsigned)(B * n)), dim3(T),
         [&] { mlmc::k_nodal_k_split(k0.data(), n, 1, n, B, kns.data()); });
  auto knsb = from_split(kns, perm);
  out.insert(out.end(), knp.begin(), knp.end());
  out.insert(out.end(), knsb.begin(), knsb.end());
  FILE* fo = std::fopen(argv[6], "wb");
  std::fwrite(out.data(), sizeof(float), out.size(), fo);
  std::fclose(fo);
  return 0;
}

static int split64(char** argv) {
  const int n = std::atoi(argv[2]), B = std::atoi(argv[3]), nc = (n + 1) / 2;
  const size_t n3 = (size_t)n * n * n, nc3 = (size_t)nc * nc * nc;
  FILE* fi = std::fopen(argv[4], "rb");
  FILE* fp = std::fopen(argv[5], "rb");
  if (!fi || !fp) return 3;
  auto k0 = readv<double>(fi, B * n3), g = readv<double>(fi, B * n3), u = readv<double>(fi, B * n3);
  auto ec = readv<double>(fi, B * nc3), r = readv<double>(fi, B * n3);
  auto perm = readv<int64_t>(fp, B * n3), permc = readv<int64_t>(fp, B * nc3);
  std::fclose(fi);
  std::fclose(fp);
  const double nan = std::numeric_limits<double>::quiet_NaN();
  const size_t ns = mlmc::split_elems(n), nsc = mlmc::split_elems(nc);
  auto to_split = [&](const std::vector<double>& a, const std::vector<int64_t>& pm, size_t total) {
    std::vector<double> b(total, nan);  // slots without a node stay NaN: reading one poisons the result
    for (size_t i = 0; i < a.size(); ++i) b[pm[i]] = a[i];
    return b;
  };
  auto from_split = [&](const std::vector<double>& b, const std::vector<int64_t>& pm) {
    std::vector<double> a(pm.size());
    for (size_t i = 0; i < pm.size(); ++i) a[i] = b[pm[i]];
    return a;
  };
  std::vector<double> out;
  auto emit = [&](const std::vector<double>& plain, const std::vector<double>& split_back) {
    out.insert(out.end(), plain.begin(), plain.end());
    out.insert(out.end(), split_back.begin(), split_back.end());
  };
  const unsigned T = 64;
  const dim3 pgrid((unsigned)((n * n + T - 1) / T), (unsigned)(B * n));
  // faces and diagonals
  std::vector<double> Kx(B * n3, nan), Ky(B * n3, nan), Kz(B * n3, nan), D(B * n3, nan), Di(B * n3, nan);
  std::vector<double> sKx(B * ns, nan), sKy(B * ns, nan), sKz(B * ns, nan), sD(B * ns, nan), sDi(B * ns, nan);
  launch(pgrid, dim3(T), [&] { mlmc::k_faces<double>(k0.data(), n, 1, n, B, Kx.data(), Ky.data(), Kz.data()); });
  launch(pgrid, dim3(T), [&] { mlmc::k_faces_split(k0.data(), n, 1, n, B, sKx.data(), sKy.data(), sKz.data()); });
  launch(pgrid, dim3(T), [&] {
    mlmc::k_diag<double, double>(n, B, Kx.data(), Ky.data(), Kz.data(), D.data(), Di.data());
  });
  launch(pgrid, dim3(T), [&] {
    mlmc::k_diag_split(n, B, sKx.data(), sKy.data(), sKz.data(), sD.data(), sDi.data());
  });
  emit(Kx, from_split(sKx, perm));
  emit(Ky, from_split(sKy, perm));
  emit(Kz, from_split(sKz, perm));
  emit(D, from_split(sD, perm));
  emit(Di, from_split(sDi, perm));
  // a red and a black pass (u and g enter the split storage through the copy kernel)
  const int m = n - 2, half = (n - 1) / 2, P = mlmc::split_pitch(n);
  std::vector<double> up = u, us(B * ns, nan), gs(B * ns, nan);
  launch(pgrid, dim3(T), [&] { mlmc::k_split_copy<double, true>(n, B, u.data(), us.data()); });
  launch(pgrid, dim3(T), [&] { mlmc::k_split_copy<double, true>(n, B, g.data(), gs.data()); });
  for (int c = 0; c < 2; ++c) {
    launch(dim3((unsigned)((m * half + T - 1) / T), (unsigned)(B * m)), dim3(T), [&] {
      mlmc::k_rbgs<double>(c, n, B, Kx.data(), Ky.data(), Kz.data(), Di.data(), g.data(), up.data(), nullptr);
    });
    MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)((m * (P / 2) + 127) / 128), (unsigned)m, (unsigned)B), dim3(128), [&] {
      mlmc::k_rbgs_split64<LG>(c, sKx.data(), sKy.data(), sKz.data(), sDi.data(), gs.data(), us.data(), nullptr);
    }));
  }
  emit(up, from_split(us, perm));
  // the residual of the swept iterate (one z-slab per column)
  std::vector<double> rp(B * n3, nan), rss(B * ns, 0.0);
  launch(dim3((unsigned)((n * n + 127) / 128), 1, (unsigned)B), dim3(128), [&] {
    mlmc::k_residual_z<double, double, double, double>(n, n - 2, Kx.data(), Ky.data(), Kz.data(), D.data(), g.data(),
                                                       up.data(), rp.data(), nullptr, nullptr);
  });
  MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)((m * (P / 2) + 127) / 128), (unsigned)(2 * m), (unsigned)B), dim3(128), [&] {
    mlmc::k_residual_split64<LG>(sKx.data(), sKy.data(), sKz.data(), sD.data(), gs.data(), us.data(), rss.data(),
                                 nullptr);
  }));
  emit(rp, from_split(rss, perm));  // the split residual leaves boundary slots unwritten (zero here)
  // the trilinear correction: k_prolong against the block form (one thread per coarse
  // cell), plain and split, and in FP32
  std::vector<double> pp = u, ecs = to_split(ec, permc, B * nsc);
  launch(dim3((unsigned)((m * (n - 1) + T - 1) / T), (unsigned)(B * m)), dim3(T),
         [&] { mlmc::k_prolong<double>(n, B, ec.data(), pp.data(), nullptr); });
  // the block form (one thread per coarse cell), plain and split, and in FP32
  const int mc = nc - 1;
  std::vector<double> pb = u, pbs = to_split(u, perm, B * ns);
  launch(dim3((unsigned)((mc * mc + 127) / 128), (unsigned)(B * mc)), dim3(128),
         [&] { mlmc::k_prolong_blk<double>(n, B, ec.data(), pb.data(), nullptr); });
  MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)((mc * mc + 127) / 128), (unsigned)mc, (unsigned)B), dim3(128), [&] {
    mlmc::k_prolong_blk_split<LG, double>(ecs.data(), pbs.data(), nullptr);
  }));
  emit(pp, pb);
  emit(pp, from_split(pbs, perm));
  std::vector<float> uf(u.begin(), u.end()), ecf(ec.begin(), ec.end());
  std::vector<float> pf = uf, pbf = uf;
  launch(dim3((unsigned)((m * (n - 1) + T - 1) / T), (unsigned)(B * m)), dim3(T),
         [&] { mlmc::k_prolong<float>(n, B, ecf.data(), pf.data(), nullptr); });
  launch(dim3((unsigned)((mc * mc + 127) / 128), (unsigned)(B * mc)), dim3(128),
         [&] { mlmc::k_prolong_blk<float>(n, B, ecf.data(), pbf.data(), nullptr); });
  emit(std::vector<double>(pf.begin(), pf.end()), std::vector<double>(pbf.begin(), pbf.end()));
  // full weighting into the plain and the split coarse storage
  std::vector<double> gcp(B * nc3, 0.0), gcs(B * nsc, 0.0), r_s = to_split(r, perm, B * ns);
  const int hc = nc - 1;
  launch(dim3((unsigned)(((nc - 2) * hc + T - 1) / T), (unsigned)(B * (nc - 2))), dim3(T),
         [&] { mlmc::k_restrict<double, false>(n, B, r.data(), gcp.data(), nullptr); });
  MLMC_SPLIT_DISPATCH(n, launch(dim3((unsigned)(((nc - 2) * (nc - 2) + 127) / 128), (unsigned)(nc - 2), (unsigned)B),
                                dim3(128), [&] { mlmc::k_restrict_split<LG, double>(r_s.data(), gcs.data(), nullptr); }));
  emit(gcp, from_split(gcs, permc));
  // plain -> split -> plain
  std::vector<double> back(B * n3, nan);
  launch(pgrid, dim3(T), [&] { mlmc::k_split_copy<double, false>(n, B, us.data(), back.data()); });
  emit(from_split(us, perm), back);
  // the P1 transfers of the finite-element path, plain and colour-split
  {
    std::vector<double> pl = u, ps1 = to_split(u, perm, B * ns);
    const std::vector<double> ecs1 = to_split(ec, permc, B * nsc);
    launch(dim3((unsigned)((m * m + T - 1) / T), (unsigned)(B * m)), dim3(T),
           [&] { mlmc::k_prolong_p1<double, false>(n, B, ec.data(), pl.data(), nullptr); });
    launch(dim3((unsigned)((m * m + T - 1) / T), (unsigned)(B * m)), dim3(T),
           [&] { mlmc::k_prolong_p1<double, true>(n, B, ecs1.data(), ps1.data(), nullptr); });
    emit(pl, from_split(ps1, perm));
    const int mc = nc - 2;
    std::vector<double> gp(B * nc3, 0.0), gsp(B * nsc, 0.0);
    const std::vector<double> rsp = to_split(r, perm, B * ns);
    launch(dim3((unsigned)((mc * mc + T - 1) / T), (unsigned)(B * mc)), dim3(T),
           [&] { mlmc::k_restrict_p1<double, false>(n, B, r.data(), gp.data(), nullptr); });
    launch(dim3((unsigned)((mc * mc + T - 1) / T), (unsigned)(B * mc)), dim3(T),
           [&] { mlmc::k_restrict_p1<double, true>(n, B, rsp.data(), gsp.data(), nullptr); });
    emit(gp, from_split(gsp, permc));
  }
  FILE* fo = std::fopen(argv[6], "wb");
  std::fwrite(out.data(), sizeof(double), out.size(), fo);
  std::fclose(fo);
  return 0;
}
