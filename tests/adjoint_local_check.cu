// Host check of the adjoint's reverse-mode local adjoints (revise_flux_adj,
// side_rec_adj, own_terms_adj, friction_cell_adj) against forward-mode dual
// numbers through the templated point functions they differentiate, on random
// states that cover the dry, partially wet, thin-limit and HLL-regime
// branches.  tests/test_adjoint_local_host.py builds it with nvcc from the
// device functions of paper_2010_02003_gb300/csrc/dg2_adj.cu (compiled for
// the host) and runs it; exit status 0 = every gradient within 1e-9.
#include <cmath>
#include <cstdio>
#include <random>
#include "adj_head.inc"
int run() {
  std::mt19937_64 rng(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  Prob p{};
  p.g = 9.80665; p.tol = 1e-5; p.wd = 1; p.inv_dx = 0.5; p.inv_dy = 0.5;
  double worst_face = 0, worst_side = 0, worst_own = 0, worst_fric = 0;
  for (int it = 0; it < 200000; ++it) {
    // random records (some partially wet, some dry)
    RecT<real> Ra, Rb;
    auto mk = [&](RecT<real>& r) {
      r.h = U(rng) * 0.5 + (U(rng) > -0.6 ? 0.3 : -0.2);
      r.u = U(rng); r.v = U(rng);
      r.hs = r.h > 0 ? r.h * (1.0 + 0.3 * std::fabs(U(rng))) : 0.0;
      r.zf = U(rng); r.pw = U(rng) > 0.3;
    };
    mk(Ra); mk(Rb);
    const bool y = U(rng) > 0;
    real wF[3] = {U(rng), U(rng), U(rng)}, wha = U(rng), wza = U(rng), whb = U(rng), wzb = U(rng);
    real ga[4] = {0, 0, 0, 0}, gb[4] = {0, 0, 0, 0};
    revise_flux_adj(Ra, Rb, y, p.g, p.tol, wF, wha, wza, whb, wzb, ga, gb);
    RecT<Dual<8>> Da, Db;
    Da.h = var<8>(Ra.h, 0); Da.u = var<8>(Ra.u, 1); Da.v = var<8>(Ra.v, 2); Da.hs = var<8>(Ra.hs, 3);
    Da.zf = Ra.zf; Da.pw = Ra.pw;
    Db.h = var<8>(Rb.h, 4); Db.u = var<8>(Rb.u, 5); Db.v = var<8>(Rb.v, 6); Db.hs = var<8>(Rb.hs, 7);
    Db.zf = Rb.zf; Db.pw = Rb.pw;
    LimT<Dual<8>> ra, rb; Dual<8> ha, za, hb, zb;
    revise_face_t(Da, Db, p.tol, ra, rb, ha, za, hb, zb);
    const F3T<Dual<8>> F = flux_face(ra, rb, y, p.g, p.tol);
    for (int k = 0; k < 8; ++k) {
      const double ref = wF[0] * F.h.d[k] + wF[1] * F.x.d[k] + wF[2] * F.y.d[k] + wha * ha.d[k] +
                         wza * za.d[k] + whb * hb.d[k] + wzb * zb.d[k];
      const double got = k < 4 ? ga[k] : gb[k - 4];
      const double e = std::fabs(got - ref) / (1e-12 + std::fabs(ref));
      if (e > worst_face) worst_face = e;
      if (e > 1e-9) { printf("face it %d k %d ref %g got %g\n", it, k, ref, got); return 1; }
    }
    // side record
    real h4[4] = {U(rng) * 0.3 + 0.1, U(rng) * 0.3 + 0.1, U(rng) * 0.3 + 0.1, U(rng) * 0.3 + 0.1};
    const real qx = U(rng), qy = U(rng), h0v = 0.5 * (h4[0] + h4[1]) + 0.01 * U(rng);
    const int fo = it % 4;
    real grw[4] = {U(rng), U(rng), U(rng), U(rng)}, g6[6];
    side_rec_adj(p, h4, qx, qy, h0v, fo, grw, g6);
    Dual<6> D4[4];
    for (int q = 0; q < 4; ++q) D4[q] = var<6>(h4[q], q);
    const RecT<Dual<6>> R = side_rec(p, D4, var<6>(qx, 4), var<6>(qy, 5), h0v, fo, 0.0);
    for (int k = 0; k < 6; ++k) {
      const double ref = grw[0] * R.h.d[k] + grw[1] * R.u.d[k] + grw[2] * R.v.d[k] + grw[3] * R.hs.d[k];
      const double e = std::fabs(g6[k] - ref) / (1e-12 + std::fabs(ref));
      if (e > worst_side) worst_side = e;
      if (e > 1e-9) { printf("side it %d k %d ref %g got %g\n", it, k, ref, g6[k]); return 1; }
    }
    // own terms
    real hs[4], zs[4], uu[4], vv[4], mu[9];
    for (int f = 0; f < 4; ++f) { hs[f] = std::fabs(U(rng)) * 0.5; zs[f] = U(rng); uu[f] = U(rng); vv[f] = U(rng); }
    for (int k = 0; k < 9; ++k) mu[k] = U(rng);
    real g_hs[4], g_zs[4], g_u[4], g_v[4];
    own_terms_adj(p, hs, zs, uu, vv, mu, g_hs, g_zs, g_u, g_v);
    {
      Dual<16> H[4], Z[4], Uu[4], V[4], L[9];
      for (int f = 0; f < 4; ++f) { H[f] = var<16>(hs[f], f); Z[f] = var<16>(zs[f], 4 + f); Uu[f] = var<16>(uu[f], 8 + f); V[f] = var<16>(vv[f], 12 + f); }
      own_terms<Dual<16>>(p, H, Z, Uu, V, L);
      for (int q = 0; q < 16; ++q) {
        double ref = 0; for (int k = 0; k < 9; ++k) ref += mu[k] * L[k].d[q];
        const double got = q < 4 ? g_hs[q] : q < 8 ? g_zs[q - 4] : q < 12 ? g_u[q - 8] : g_v[q - 12];
        const double e = std::fabs(got - ref) / (1e-12 + std::fabs(ref));
        if (e > worst_own) worst_own = e;
        if (e > 1e-9) { printf("own it %d q %d ref %g got %g\n", it, q, ref, got); return 1; }
      }
    }
    // friction
    real m[9], ls[9], gm[9], gn;
    for (int k = 0; k < 9; ++k) { m[k] = U(rng) * 0.3; ls[k] = U(rng); }
    m[0] = std::fabs(m[0]) + 0.05;
    const real nman = 0.03 + 0.02 * std::fabs(U(rng)), dt = 0.1;
    friction_cell_adj(m, nman, dt, p.g, p.tol, ls, gm, gn);
    {
      Dual<10> M[9], O[9];
      for (int k = 0; k < 9; ++k) M[k] = var<10>(m[k], k);
      friction_cell<Dual<10>>(M, var<10>(nman, 9), dt, p.g, p.tol, O);
      for (int q = 0; q < 10; ++q) {
        double ref = 0; for (int k = 0; k < 9; ++k) ref += ls[k] * O[k].d[q];
        const double got = q < 9 ? gm[q] : gn;
        const double e = std::fabs(got - ref) / (1e-12 + std::fabs(ref));
        if (e > worst_fric) worst_fric = e;
        if (e > 1e-9) { printf("fric it %d q %d ref %g got %g\n", it, q, ref, got); return 1; }
      }
    }
  }
  printf("worst relative: face %.2e side %.2e own %.2e friction %.2e\n", worst_face, worst_side, worst_own, worst_fric);
  return 0;
}
}  // namespace adj
}  // namespace dg2
int main() { return dg2::adj::run(); }
