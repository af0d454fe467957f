// opcount.cpp -- counts the floating-point operations of the oracle's scheme.
//
// TEST INFRASTRUCTURE ONLY (measurement): compiles dg2_oracle.c unchanged as
// C++ with its `real` type set to a scalar that counts every addition,
// subtraction, multiplication, division, square root and cube root it takes
// part in, then steps a fully wet, moving grid and reports operations per cell
// per RK2 step (printed face revision; see below).  The oracle evaluates each
// interior face flux twice (once from
// each side); the cost of one HLL evaluation is measured separately so the
// once-per-face figure is formed: total - 4 HLL evaluations per cell-step.
//
// Build/run: g++ -O1 -std=c++17 -o opcount oracle/opcount.cpp && ./opcount
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace opc {
struct Stats {
  long long add = 0, mul = 0, div = 0, sqrt = 0, cbrt = 0;
};
Stats total;
inline void count_add() { total.add++; }
inline void count_mul() { total.mul++; }
inline void count_div() { total.div++; }
inline void count_sqrt() { total.sqrt++; }
inline void count_cbrt() { total.cbrt++; }
}  // namespace opc

struct Cnt {
  double v;
  Cnt() : v(0.0) {}
  Cnt(double x) : v(x) {}
  operator double() const { return v; }
};
#define BIN(op, counter)                                                               \
  inline Cnt operator op(Cnt a, Cnt b) { opc::counter(); return Cnt(a.v op b.v); }     \
  inline Cnt operator op(Cnt a, double b) { opc::counter(); return Cnt(a.v op b); }    \
  inline Cnt operator op(double a, Cnt b) { opc::counter(); return Cnt(a op b.v); }    \
  inline Cnt operator op(Cnt a, int b) { opc::counter(); return Cnt(a.v op b); }         \
  inline Cnt operator op(int a, Cnt b) { opc::counter(); return Cnt(a op b.v); }
BIN(+, count_add)
BIN(-, count_add)
BIN(*, count_mul)
BIN(/, count_div)
#undef BIN
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
#define CMP(op)                                                        \
  inline bool operator op(Cnt a, Cnt b) { return a.v op b.v; }         \
  inline bool operator op(Cnt a, double b) { return a.v op b; }        \
  inline bool operator op(double a, Cnt b) { return a op b.v; }
CMP(<) CMP(>) CMP(<=) CMP(>=) CMP(==) CMP(!=)
#undef CMP
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline Cnt sqrt(Cnt a) { opc::count_sqrt(); return Cnt(std::sqrt(a.v)); }
inline Cnt cbrt(Cnt a) { opc::count_cbrt(); return Cnt(std::cbrt(a.v)); }
inline Cnt fabs(Cnt a) { return Cnt(std::fabs(a.v)); }
using std::sqrt;
using std::cbrt;
using std::fabs;
using std::floor;

#define ORC_REAL Cnt
#include "dg2_oracle.c"

int main(int argc, char** argv) {
  const int n = argc > 1 ? atoi(argv[1]) : 64;
  const int limiter = argc > 2 ? atoi(argv[2]) : 0;
  int bc[4] = {0, 0, 0, 0};
  orc_t* o = orc_create(n, n, 2.0, 2.0, 9.80665, 0.3, 1e-5, 10.0, 1.0, limiter, bc);
  // the printed face revision: on fully wet flow the default revision does the
  // same arithmetic plus one multiplication per face limit (its thin-limit
  // threshold h0 / 10), while the oracle's statement of it rebuilds every
  // neighbour's four face records per cell, which is not work of the scheme
  orc_set_wetdry(o, 0);
  // fully wet, moving: tilted free surface over a wavy bed, uniform Manning n
  double* zc = (double*)malloc(sizeof(double) * (n + 1) * (n + 1));
  double* ec = (double*)malloc(sizeof(double) * (n + 1) * (n + 1));
  for (int j = 0; j <= n; ++j)
    for (int i = 0; i <= n; ++i) {
      zc[j * (n + 1) + i] = 0.2 * std::sin(0.3 * i) * std::cos(0.2 * j);
      ec[j * (n + 1) + i] = 2.0 - 0.01 * i + 0.005 * j;
    }
  orc_set_dem(o, zc, nullptr, 0.04, ec);
  for (int k = 0; k < 3; ++k) orc_step(o, orc_cfl_dt(o));   // develop velocities
  opc::total = opc::Stats();
  const int steps = 5;
  for (int k = 0; k < steps; ++k) orc_step(o, 0.01);
  const double cells = (double)n * n * steps;
  auto pr = [&](const char* name, const opc::Stats& s) {
    printf("%-6s add %8.1f mul %8.1f div %6.1f sqrt %5.1f cbrt %5.1f  flops %8.1f\n", name,
           s.add / cells, s.mul / cells, s.div / cells, s.sqrt / cells, s.cbrt / cells,
           (s.add + s.mul + s.div + s.sqrt + s.cbrt) / cells);
  };
  pr("total", opc::total);
  // ops of one HLL evaluation between two wet, moving states (the general branch)
  const opc::Stats before = opc::total;
  const int calls = 1000;
  for (int k = 0; k < calls; ++k) {
    double l[3] = {1.0 + 1e-3 * k, 0.3, -0.1}, r[3] = {0.9, 0.2 + 1e-4 * k, 0.05}, f[3];
    orc_hll(o, k & 1, l, r, f);
  }
  opc::Stats per = opc::total;
  per.add -= before.add; per.mul -= before.mul; per.div -= before.div;
  per.sqrt -= before.sqrt; per.cbrt -= before.cbrt;
  const double pc = 1.0 / calls;
  printf("hll/call add %.1f mul %.1f div %.1f sqrt %.1f\n", per.add * pc, per.mul * pc,
         per.div * pc, per.sqrt * pc);
  // the oracle evaluates 8 face fluxes per cell-step (4 faces x 2 stages), each
  // interior face twice; once per face is 4 evaluations per cell-step
  opc::Stats once = before;
  once.add -= (long long)(4 * cells * per.add * pc); once.mul -= (long long)(4 * cells * per.mul * pc);
  once.div -= (long long)(4 * cells * per.div * pc); once.sqrt -= (long long)(4 * cells * per.sqrt * pc);
  pr("once", once);

  // per routine, through the oracle's exported entry points (one call each)
  const double N1 = (double)n * n;
  std::vector<double> U((size_t)9 * n * n), L((size_t)9 * n * n), U2((size_t)9 * n * n);
  orc_get_state(o, U.data(), nullptr);
  auto span = [&](const char* name, auto fn, double hll_calls_to_drop) {
    const opc::Stats b0 = opc::total;
    fn();
    opc::Stats d = opc::total;
    d.add -= b0.add; d.mul -= b0.mul; d.div -= b0.div; d.sqrt -= b0.sqrt; d.cbrt -= b0.cbrt;
    d.add -= (long long)(hll_calls_to_drop * N1 * per.add * pc);
    d.mul -= (long long)(hll_calls_to_drop * N1 * per.mul * pc);
    d.div -= (long long)(hll_calls_to_drop * N1 * per.div * pc);
    d.sqrt -= (long long)(hll_calls_to_drop * N1 * per.sqrt * pc);
    const double c1 = 1.0 / N1;
    printf("%-9s add %7.1f mul %7.1f div %6.1f sqrt %5.1f cbrt %4.1f  flops %7.1f per cell\n", name,
           d.add * c1, d.mul * c1, d.div * c1, d.sqrt * c1, d.cbrt * c1,
           (d.add + d.mul + d.div + d.sqrt + d.cbrt) * c1);
  };
  span("friction", [&] { orc_friction(o, U.data(), 0.01); }, 0.0);
  span("operator", [&] { orc_operator(o, U.data(), 0.0, L.data()); }, 2.0);
  span("limiter", [&] { orc_limit(o, U.data(), U2.data()); }, 0.0);
  orc_destroy(o);
  return 0;
}
