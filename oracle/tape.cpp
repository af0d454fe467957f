// tape.cpp -- reverse-mode (taped) derivatives of the oracle's DG2 run.
//
// TEST INFRASTRUCTURE ONLY: compiles dg2_oracle.c unchanged as C++ with its
// `real` type set to a scalar that records every operation on a tape (value,
// operand nodes, local partial derivatives).  Running the oracle's steps and
// the gauge misfit in that type and sweeping the tape backwards gives the
// exact derivatives of the oracle's own computation: every branch (wet-dry,
// revision, HLL regime, ghost) is the one its values take.  Conventions where
// a function has no derivative: sqrt and cbrt of 0 and |.| at 0 get 0.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -fPIC -shared -o liboracle_tape.so oracle/tape.cpp
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace tp {
struct Node {
  int a, b;
  double da, db;
};
std::vector<Node> nodes;  // node 0: constants (never propagated)
inline int push(int a, double da, int b, double db) {
  if (a == 0 && b == 0) return 0;
  nodes.push_back(Node{a, b, da, db});
  return (int)nodes.size() - 1;
}
}  // namespace tp

struct Tape {
  double v;
  int id;
  Tape() : v(0.0), id(0) {}
  Tape(double x) : v(x), id(0) {}
  Tape(double x, int i) : v(x), id(i) {}
  operator double() const { return v; }
};

inline Tape operator+(Tape a, Tape b) { return Tape(a.v + b.v, tp::push(a.id, 1.0, b.id, 1.0)); }
inline Tape operator-(Tape a, Tape b) { return Tape(a.v - b.v, tp::push(a.id, 1.0, b.id, -1.0)); }
inline Tape operator*(Tape a, Tape b) { return Tape(a.v * b.v, tp::push(a.id, b.v, b.id, a.v)); }
inline Tape operator/(Tape a, Tape b) {
  const double r = a.v / b.v;
  return Tape(r, tp::push(a.id, 1.0 / b.v, b.id, -r / b.v));
}
inline Tape operator-(Tape a) { return Tape(-a.v, tp::push(a.id, -1.0, 0, 0.0)); }
#define MIXED(op)                                                     \
  inline Tape operator op(Tape a, double b) { return a op Tape(b); }  \
  inline Tape operator op(double a, Tape b) { return Tape(a) op b; }  \
  inline Tape operator op(Tape a, int b) { return a op Tape(b); }     \
  inline Tape operator op(int a, Tape b) { return Tape(a) op b; }
MIXED(+) MIXED(-) MIXED(*) MIXED(/)
#undef MIXED
#define CMP(op)                                                        \
  inline bool operator op(Tape a, Tape b) { return a.v op b.v; }       \
  inline bool operator op(Tape a, double b) { return a.v op b; }       \
  inline bool operator op(double a, Tape b) { return a op b.v; }
CMP(<) CMP(>) CMP(<=) CMP(>=) CMP(==) CMP(!=)
#undef CMP
inline Tape& operator+=(Tape& a, Tape b) { a = a + b; return a; }
inline Tape& operator-=(Tape& a, Tape b) { a = a - b; return a; }
inline Tape sqrt(Tape a) {
  const double r = std::sqrt(a.v);
  return Tape(r, tp::push(a.id, r > 0.0 ? 0.5 / r : 0.0, 0, 0.0));
}
inline Tape cbrt(Tape a) {
  const double r = std::cbrt(a.v);
  return Tape(r, tp::push(a.id, r != 0.0 ? 1.0 / (3.0 * r * r) : 0.0, 0, 0.0));
}
inline Tape fabs(Tape a) {
  return Tape(std::fabs(a.v), tp::push(a.id, a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0), 0, 0.0));
}
using std::sqrt;
using std::cbrt;
using std::fabs;
using std::floor;

#define ORC_REAL Tape
#include "dg2_oracle.c"

extern "C" {

// Loss J = sum_s sum_g (h_g(U after samp_step[s] steps) - obs[s][g])^2 of the
// oracle run of nsteps steps of sizes dts from the DEM / water / Manning /
// inflow given, and its derivatives with respect to the Manning n of every
// cell (grad_n[ny*nx]) and the inflow knot discharges (grad_q[nk]).
double orc_tape_gradient(int nx, int ny, double dx, double dy, double g, double cfl, double tol,
                         double ds, double dt_max, int limiter, int wd, const int *bc,
                         const double *z_corner, const double *eta_corner, const double *manning,
                         int edge, double s0, double len, const double *tk, const double *qk,
                         int nk, int nsteps, const double *dts, int nsamp, const int *samp_step,
                         int ngauge, const double *gxy, const double *obs, double *grad_n,
                         double *grad_q)
{
    tp::nodes.clear();
    tp::nodes.push_back(tp::Node{0, 0, 0.0, 0.0});
    orc_t *o = orc_create(nx, ny, dx, dy, g, cfl, tol, ds, dt_max, limiter, bc);
    const size_t N = (size_t)nx * ny;
    orc_set_wetdry(o, wd);
    orc_set_dem(o, z_corner, manning, 0.0, eta_corner);
    // the parameters become tape variables
    std::vector<int> nid(N), qid(nk > 0 ? nk : 0);
    for (size_t c = 0; c < N; ++c) {
        nid[c] = tp::push(-1, 0.0, 0, 0.0);   // a leaf: parent -1 is never followed
        o->nm[c] = Tape(manning[c], nid[c]);
    }
    if (edge >= 0 && nk > 0) {
        orc_add_inflow(o, edge, s0, len, tk, qk, nk);
        for (int k = 0; k < nk; ++k) {
            qid[k] = tp::push(-1, 0.0, 0, 0.0);
            o->in[0].qk[k] = Tape(qk[k], qid[k]);
        }
    }
    Tape J(0.0);
    auto sample = [&](int k) {
        for (int s = 0; s < nsamp; ++s) {
            if (samp_step[s] != k) continue;
            for (int q = 0; q < ngauge; ++q) {
                const double x = gxy[2 * q], y = gxy[2 * q + 1];
                int i = (int)std::floor(x / dx), j = (int)std::floor(y / dy);
                if (i < 0) i = 0;
                if (i >= nx) i = nx - 1;
                if (j < 0) j = 0;
                if (j >= ny) j = ny - 1;
                const size_t c = (size_t)j * nx + i;
                const double xi = (x - (i + 0.5) * dx) / (0.5 * dx), et = (y - (j + 0.5) * dy) / (0.5 * dy);
                Tape h = o->U[c] + xi * o->U[N + c] + et * o->U[2 * N + c];
                if (!(h > 0.0)) h = Tape(0.0);
                const Tape r = h - obs[(size_t)s * ngauge + q];
                J = J + r * r;
            }
        }
    };
    sample(0);
    for (int k = 0; k < nsteps; ++k) {
        orc_step(o, dts[k]);
        sample(k + 1);
    }
    // reverse sweep
    std::vector<double> adj(tp::nodes.size(), 0.0);
    if (J.id > 0) adj[J.id] = 1.0;
    for (size_t n = tp::nodes.size() - 1; n > 0; --n) {
        const double w = adj[n];
        if (w == 0.0) continue;
        const tp::Node &nd = tp::nodes[n];
        if (nd.a > 0) adj[nd.a] += nd.da * w;
        if (nd.b > 0) adj[nd.b] += nd.db * w;
    }
    for (size_t c = 0; c < N; ++c) grad_n[c] = nid[c] > 0 ? adj[nid[c]] : 0.0;
    for (int k = 0; k < nk; ++k) grad_q[k] = (edge >= 0 && qid[k] > 0) ? adj[qid[k]] : 0.0;
    const double loss = J.v;
    orc_destroy(o);
    tp::nodes.clear();
    tp::nodes.shrink_to_fit();
    return loss;
}

}  // extern "C"
