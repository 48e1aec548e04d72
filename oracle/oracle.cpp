// oracle.cpp -- plain FP64 CPU oracle for one RK2 cycle of ideal MHD.
//
// TEST INFRASTRUCTURE ONLY (see oracle.h).  Written for readability against the
// paper, not for speed: plain loops over cells and faces, periodic wrap by index
// arithmetic, no blocking and no fusion.  Built with -ffp-contract=off so every
// add and multiply is rounded on its own.  The only parallel construct is an
// OpenMP loop over k-planes (it does not change any result).
//
// The arithmetic is written once as templates over the scalar type R so that the
// same code can be run with an operation-counting scalar (Counted) to measure the
// algorithmic flops of the method.
//
// Parity pins: every function here is checked by tests/test_oracle_*.py against
// closed forms (exact Riemann solution, linear-wave eigenmodes), invariants
// (conservation, div B, uniform states, symmetries) and independent formulas
// (Toro's HLLC at B = 0, characteristic speeds of the flux Jacobian).
#include "oracle.h"

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Operation-counting scalar (single-threaded use only).  Each add/sub, mul, div and
// square root of a Counted value is tallied, and so is each comparison; negation and
// absolute value are sign operations and are not.  The tally is kept per part of the
// method (ORA_PART_* of oracle.h), so that work this plain code repeats for clarity --
// each cell's van Leer slope is formed for both faces that use it, each cell-centre EMF
// for the four edges around it -- can be told apart from the method's own work.
// ---------------------------------------------------------------------------
struct Tally {
  double add = 0, mul = 0, div = 0, sqrt = 0, cmp = 0;
};
Tally g_parts[ORA_NUM_PARTS];
int g_part = ORA_PART_DT;
inline Tally& tally() { return g_parts[g_part]; }
void reset_tally() {
  for (int p = 0; p < ORA_NUM_PARTS; ++p) g_parts[p] = Tally();
  g_part = ORA_PART_DT;
}

struct Counted {
  double v;
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}  // NOLINT: implicit on purpose, constants enter as doubles
};
inline Counted operator+(Counted a, Counted b) { tally().add += 1; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { tally().add += 1; return Counted(a.v - b.v); }
inline Counted operator*(Counted a, Counted b) { tally().mul += 1; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { tally().div += 1; return Counted(a.v / b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline bool operator<(Counted a, Counted b) { tally().cmp += 1; return a.v < b.v; }
inline bool operator>(Counted a, Counted b) { tally().cmp += 1; return a.v > b.v; }
inline bool operator<=(Counted a, Counted b) { tally().cmp += 1; return a.v <= b.v; }
inline bool operator>=(Counted a, Counted b) { tally().cmp += 1; return a.v >= b.v; }
inline bool operator==(Counted a, Counted b) { tally().cmp += 1; return a.v == b.v; }
inline Counted sq_root(Counted a) { tally().sqrt += 1; return Counted(std::sqrt(a.v)); }
inline Counted absval(Counted a) { return Counted(std::fabs(a.v)); }
inline double value(Counted a) { return a.v; }

inline double sq_root(double a) { return std::sqrt(a); }
inline double absval(double a) { return std::fabs(a); }
inline double value(double a) { return a; }

template <class R> constexpr bool kPar = std::is_same<R, double>::value;

// Sets the part that counted operations are tallied under (no effect for plain doubles).
template <class R> inline void in_part(int part) {
  if constexpr (std::is_same<R, Counted>::value) g_part = part;
}

template <class R> inline R rmax(R a, R b) { return (a < b) ? b : a; }
template <class R> inline R rmin(R a, R b) { return (b < a) ? b : a; }

// ---------------------------------------------------------------------------
// Grid helpers.  Direction d = 0, 1, 2 for x, y, z.
// ---------------------------------------------------------------------------
struct Grid {
  int n[3];
  double dl[3];
  bool active[3];  // a direction with a single cell is not integrated
  long ncell;
};

Grid make_grid(const ora_grid* g) {
  Grid G;
  G.n[0] = g->nx; G.n[1] = g->ny; G.n[2] = g->nz;
  G.dl[0] = g->lx / g->nx; G.dl[1] = g->ly / g->ny; G.dl[2] = g->lz / g->nz;
  for (int d = 0; d < 3; ++d) G.active[d] = G.n[d] > 1;
  G.ncell = (long)g->nx * g->ny * g->nz;
  return G;
}

bool grid_ok(const ora_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nz >= 1 && g->lx > 0 && g->ly > 0 && g->lz > 0;
}

inline int wrap(int i, int n) { return ((i % n) + n) % n; }

// flat index of cell (i, j, k), periodic
inline long at(const Grid& G, int i, int j, int k) {
  return ((long)wrap(k, G.n[2]) * G.n[1] + wrap(j, G.n[1])) * G.n[0] + wrap(i, G.n[0]);
}
// flat index of cell (i, j, k) + s e_d
inline long shift(const Grid& G, int i, int j, int k, int d, int s) {
  int c[3] = {i, j, k};
  c[d] += s;
  return at(G, c[0], c[1], c[2]);
}
inline long shift2(const Grid& G, int i, int j, int k, int d1, int s1, int d2, int s2) {
  int c[3] = {i, j, k};
  c[d1] += s1;
  c[d2] += s2;
  return at(G, c[0], c[1], c[2]);
}

// Field indices of the conserved set and of the primitive set.
enum { RHO = 0, MX = 1, MY = 2, MZ = 3, EN = 4, BX = 5, BY = 6, BZ = 7 };
enum { PR = 4 };  // pressure slot in the primitive set (rho, vx, vy, vz, P, Bcx, Bcy, Bcz)

// ---------------------------------------------------------------------------
// Primitive recovery (Sec. 2.1 definitions: E = e + rho v^2/2 + B^2/2, e = P/(gamma-1)).
// Cell-centre B is the arithmetic mean of the two face values bounding the cell.
// v = m * (1/rho).  No floors: a non-positive density or pressure is an error.
// ---------------------------------------------------------------------------
template <class R>
int prims(const Grid& G, double gamma, const std::vector<R>* U, std::vector<R>* W, long* bad) {
  in_part<R>(ORA_PART_PRIMS);
  long first_bad = G.ncell;
#pragma omp parallel for reduction(min : first_bad) if (kPar<R>)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        const R rho = U[RHO][p];
        const R inv_rho = R(1.0) / rho;
        const R vx = U[MX][p] * inv_rho;
        const R vy = U[MY][p] * inv_rho;
        const R vz = U[MZ][p] * inv_rho;
        const R bx = R(0.5) * (U[BX][p] + U[BX][shift(G, i, j, k, 0, 1)]);
        const R by = R(0.5) * (U[BY][p] + U[BY][shift(G, i, j, k, 1, 1)]);
        const R bz = R(0.5) * (U[BZ][p] + U[BZ][shift(G, i, j, k, 2, 1)]);
        const R kin = R(0.5) * rho * (vx * vx + vy * vy + vz * vz);
        const R mag = R(0.5) * (bx * bx + by * by + bz * bz);
        const R P = R(gamma - 1.0) * (U[EN][p] - kin - mag);
        W[RHO][p] = rho; W[1][p] = vx; W[2][p] = vy; W[3][p] = vz; W[PR][p] = P;
        W[5][p] = bx; W[6][p] = by; W[7][p] = bz;
        const double r = value(rho), pp = value(P);
        if (!(r > 0.0) || !(pp > 0.0) || !std::isfinite(r) || !std::isfinite(pp) ||
            !std::isfinite(value(vx)) || !std::isfinite(value(vy)) || !std::isfinite(value(vz))) {
          if (p < first_bad) first_bad = p;
        }
      }
  if (bad) *bad = (first_bad < G.ncell) ? first_bad : -1;
  return (first_bad < G.ncell) ? ORA_ENONPHYS : ORA_OK;
}

// ---------------------------------------------------------------------------
// PLM with the van Leer limiter (Sec. 2.3): harmonic mean of the one-sided
// differences when they share a sign, zero otherwise.
// ---------------------------------------------------------------------------
template <class R> R vanleer(R wm, R w0, R wp) {
  const R dL = w0 - wm;
  const R dR = wp - w0;
  const R prod = dL * dR;
  if (prod > R(0.0)) return R(2.0) * prod / (dL + dR);
  return R(0.0);
}

// ---------------------------------------------------------------------------
// Compact third-order reconstruction "LimO3" (Cada & Torrilhon 2009), the third scheme
// listed in Sec. 2.3.  With t the ratio of the difference on the far side of the cell to
// the difference toward the face, the face value is w0 + phi(t) (w_face - w0) / 2 where
//   phi(t) = max(0, min(P3(t), max(-t/2, min(2t, P3(t), 3/2)))),  P3(t) = (2 + t)/3.
// P3 alone is the unlimited third-order (parabolic) face value; the min/max chain keeps
// the face value between the neighbours (phi <= 2t, phi <= 3/2 < 2) and turns it off
// beyond a jump of the opposite sign.  The switch to P3 near smooth extrema, which the
// limiter's authors tie to a length scale, is not applied.
// ---------------------------------------------------------------------------
template <class R> R limo3_phi(R t) {
  const R p3 = (R(2.0) + t) / R(3.0);
  const R inner = rmin(rmin(R(2.0) * t, p3), R(1.5));
  return rmax(R(0.0), rmin(p3, rmax(-t / R(2.0), inner)));
}

// Face value of cell w0 on the side of w_face, with w_back its neighbour on the other side.
template <class R> R limo3_face(R w_back, R w0, R w_face) {
  const R toward = w_face - w0;
  if (value(toward) == 0.0) return w0;  // t infinite: the limit of phi(t) (w_face - w0) is 0
  const R t = (w0 - w_back) / toward;
  return w0 + limo3_phi(t) * toward / R(2.0);
}

// ---------------------------------------------------------------------------
// HLLD (Miyoshi & Kusano 2005), the magnetised HLLC counterpart named in Sec. 2.3.
// Normal = "x": state w = (rho, u, v, w, P, By, Bz), normal field bx.
// Flux ordering: (rho, m_n, m_t1, m_t2, E, Bt1, Bt2).  Pressure inside the
// momentum flux (total pressure pT = P + B^2/2).
// ---------------------------------------------------------------------------
template <class R> struct State {
  R rho, u, v, w, P, by, bz;
};

template <class R> R total_energy(const State<R>& s, R bx, double gamma) {
  return s.P / R(gamma - 1.0) + R(0.5) * s.rho * (s.u * s.u + s.v * s.v + s.w * s.w) +
         R(0.5) * (bx * bx + s.by * s.by + s.bz * s.bz);
}

// Fast magnetosonic speed along the normal.
template <class R> R fast_speed(const State<R>& s, R bx, double gamma) {
  const R gp = R(gamma) * s.P;
  const R b2 = bx * bx + s.by * s.by + s.bz * s.bz;
  const R a = gp + b2;
  const R disc = a * a - R(4.0) * gp * bx * bx;
  const R disc_pos = (disc > R(0.0)) ? disc : R(0.0);
  return sq_root((a + sq_root(disc_pos)) / (R(2.0) * s.rho));
}

template <class R> void physical_flux(const State<R>& s, R bx, R E, R F[7]) {
  const R pT = s.P + R(0.5) * (bx * bx + s.by * s.by + s.bz * s.bz);
  const R vb = s.u * bx + s.v * s.by + s.w * s.bz;
  F[0] = s.rho * s.u;
  F[1] = s.rho * s.u * s.u + pT - bx * bx;
  F[2] = s.rho * s.u * s.v - bx * s.by;
  F[3] = s.rho * s.u * s.w - bx * s.bz;
  F[4] = (E + pT) * s.u - bx * vb;
  F[5] = s.by * s.u - bx * s.v;
  F[6] = s.bz * s.u - bx * s.w;
}

// Conserved vector in flux ordering.
template <class R> void cons_vec(const State<R>& s, R E, R U[7]) {
  U[0] = s.rho;
  U[1] = s.rho * s.u;
  U[2] = s.rho * s.v;
  U[3] = s.rho * s.w;
  U[4] = E;
  U[5] = s.by;
  U[6] = s.bz;
}

template <class R>
void hlld(const State<R>& L, const State<R>& Rs, R bx, double gamma, R F[7], R* sL_out,
          R* sR_out) {
  const R EL = total_energy(L, bx, gamma);
  const R ER = total_energy(Rs, bx, gamma);
  const R bx2 = bx * bx;
  const R pTL = L.P + R(0.5) * (bx2 + L.by * L.by + L.bz * L.bz);
  const R pTR = Rs.P + R(0.5) * (bx2 + Rs.by * Rs.by + Rs.bz * Rs.bz);

  // Outer wave speeds (MK05 eq. 67).
  const R cfL = fast_speed(L, bx, gamma);
  const R cfR = fast_speed(Rs, bx, gamma);
  const R cfmax = rmax(cfL, cfR);
  const R SL = rmin(L.u, Rs.u) - cfmax;
  const R SR = rmax(L.u, Rs.u) + cfmax;
  *sL_out = SL;
  *sR_out = SR;

  R FL[7], FR[7], UL[7], UR[7];
  physical_flux(L, bx, EL, FL);
  physical_flux(Rs, bx, ER, FR);

  if (SL > R(0.0)) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q];
    return;
  }
  if (SR < R(0.0)) {
    for (int q = 0; q < 7; ++q) F[q] = FR[q];
    return;
  }
  cons_vec(L, EL, UL);
  cons_vec(Rs, ER, UR);

  // Contact speed and star total pressure (MK05 eqs. 38, 41).
  const R aL = (SL - L.u) * L.rho;   // rho_L (S_L - u_L)
  const R aR = (SR - Rs.u) * Rs.rho; // rho_R (S_R - u_R)
  const R SM = (aR * Rs.u - aL * L.u - pTR + pTL) / (aR - aL);
  const R pTs = pTL + L.rho * (SL - L.u) * (SM - L.u);

  // Single-star states (MK05 eqs. 43-48) for side alpha.
  struct Star {
    R rho, v, w, by, bz, E;
  };
  auto star = [&](const State<R>& s, R S, R E, R pT) {
    Star o;
    const R su = S - s.u;
    const R ssm = S - SM;
    o.rho = s.rho * su / ssm;
    const R D = s.rho * su * ssm - bx2;
    const R scale = absval(s.rho * su * ssm) + bx2;
    if (absval(D) <= R(1e-12) * scale) {
      // Degenerate (S = SM +- c_A with vanishing transverse field): keep the
      // transverse velocity and field unchanged.
      o.v = s.v; o.w = s.w; o.by = s.by; o.bz = s.bz;
    } else {
      o.v = s.v - bx * s.by * (SM - s.u) / D;
      o.w = s.w - bx * s.bz * (SM - s.u) / D;
      const R num = s.rho * su * su - bx2;
      o.by = s.by * num / D;
      o.bz = s.bz * num / D;
    }
    const R vb = s.u * bx + s.v * s.by + s.w * s.bz;
    const R vbs = SM * bx + o.v * o.by + o.w * o.bz;
    o.E = (su * E - pT * s.u + pTs * SM + bx * (vb - vbs)) / ssm;
    return o;
  };
  const Star sl = star(L, SL, EL, pTL);
  const Star sr = star(Rs, SR, ER, pTR);

  R UsL[7] = {sl.rho, sl.rho * SM, sl.rho * sl.v, sl.rho * sl.w, sl.E, sl.by, sl.bz};
  R UsR[7] = {sr.rho, sr.rho * SM, sr.rho * sr.v, sr.rho * sr.w, sr.E, sr.by, sr.bz};

  // Double-star states (MK05 eqs. 51, 59-63), skipped in the HLLC limit Bx -> 0.
  const R sqL = sq_root(sl.rho);
  const R sqR = sq_root(sr.rho);
  const R SsL = SM - absval(bx) / sqL;
  const R SsR = SM + absval(bx) / sqR;
  R UssL[7], UssR[7];
  if (R(0.5) * bx2 < R(1e-12) * pTs) {
    for (int q = 0; q < 7; ++q) { UssL[q] = UsL[q]; UssR[q] = UsR[q]; }
  } else {
    const R sgn = (bx < R(0.0)) ? R(-1.0) : R(1.0);
    const R inv_sum = R(1.0) / (sqL + sqR);
    const R v2 = (sqL * sl.v + sqR * sr.v + (sr.by - sl.by) * sgn) * inv_sum;
    const R w2 = (sqL * sl.w + sqR * sr.w + (sr.bz - sl.bz) * sgn) * inv_sum;
    const R by2 = (sqL * sr.by + sqR * sl.by + sqL * sqR * (sr.v - sl.v) * sgn) * inv_sum;
    const R bz2 = (sqL * sr.bz + sqR * sl.bz + sqL * sqR * (sr.w - sl.w) * sgn) * inv_sum;
    const R vb2 = SM * bx + v2 * by2 + w2 * bz2;
    const R vbL = SM * bx + sl.v * sl.by + sl.w * sl.bz;
    const R vbR = SM * bx + sr.v * sr.by + sr.w * sr.bz;
    const R E2L = sl.E - sqL * (vbL - vb2) * sgn;
    const R E2R = sr.E + sqR * (vbR - vb2) * sgn;
    UssL[0] = sl.rho; UssL[1] = sl.rho * SM; UssL[2] = sl.rho * v2; UssL[3] = sl.rho * w2;
    UssL[4] = E2L; UssL[5] = by2; UssL[6] = bz2;
    UssR[0] = sr.rho; UssR[1] = sr.rho * SM; UssR[2] = sr.rho * v2; UssR[3] = sr.rho * w2;
    UssR[4] = E2R; UssR[5] = by2; UssR[6] = bz2;
  }

  // Flux of the region that contains x/t = 0 (MK05 eq. 66).
  if (SsL >= R(0.0)) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q] + SL * (UsL[q] - UL[q]);
  } else if (SM >= R(0.0)) {
    for (int q = 0; q < 7; ++q) {
      const R FsL = FL[q] + SL * (UsL[q] - UL[q]);
      F[q] = FsL + SsL * (UssL[q] - UsL[q]);
    }
  } else if (SsR >= R(0.0)) {
    for (int q = 0; q < 7; ++q) {
      const R FsR = FR[q] + SR * (UsR[q] - UR[q]);
      F[q] = FsR + SsR * (UssR[q] - UsR[q]);
    }
  } else {
    for (int q = 0; q < 7; ++q) F[q] = FR[q] + SR * (UsR[q] - UR[q]);
  }
}

// ---------------------------------------------------------------------------
// The two more diffusive solvers of Sec. 2.3 (the paper orders its solvers from most to
// least diffusive: Rusanov, HLL, HLLC/HLLD, Roe).
//   Rusanov (Lax-Friedrichs): F = (F_L + F_R)/2 - (S_max/2)(U_R - U_L),
//     S_max = max(|u_L| + c_fL, |u_R| + c_fR).
//   HLL (Harten, Lax, van Leer; Einfeldt et al. 1991): one intermediate state between the
//     outer speeds S_L, S_R (the same estimates as HLLD):
//     F = F_L if S_L > 0, F_R if S_R < 0, else
//     F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
// Both report c = max(|S_L|, |S_R|) of the HLLD estimates for the CFL condition, so the
// time step does not depend on the solver choice.
// ---------------------------------------------------------------------------
template <class R>
void outer_speeds(const State<R>& L, const State<R>& Rs, R bx, double gamma, R* SL, R* SR,
                  R* cfL, R* cfR) {
  *cfL = fast_speed(L, bx, gamma);
  *cfR = fast_speed(Rs, bx, gamma);
  const R cfmax = rmax(*cfL, *cfR);
  *SL = rmin(L.u, Rs.u) - cfmax;
  *SR = rmax(L.u, Rs.u) + cfmax;
}

template <class R>
void rusanov(const State<R>& L, const State<R>& Rs, R bx, double gamma, R F[7], R* sL_out,
             R* sR_out) {
  R SL, SR, cfL, cfR;
  outer_speeds(L, Rs, bx, gamma, &SL, &SR, &cfL, &cfR);
  *sL_out = SL;
  *sR_out = SR;
  const R EL = total_energy(L, bx, gamma), ER = total_energy(Rs, bx, gamma);
  R FL[7], FR[7], UL[7], UR[7];
  physical_flux(L, bx, EL, FL);
  physical_flux(Rs, bx, ER, FR);
  cons_vec(L, EL, UL);
  cons_vec(Rs, ER, UR);
  const R smax = rmax(absval(L.u) + cfL, absval(Rs.u) + cfR);
  for (int q = 0; q < 7; ++q) F[q] = R(0.5) * (FL[q] + FR[q]) - R(0.5) * smax * (UR[q] - UL[q]);
}

template <class R>
void hll(const State<R>& L, const State<R>& Rs, R bx, double gamma, R F[7], R* sL_out,
         R* sR_out) {
  R SL, SR, cfL, cfR;
  outer_speeds(L, Rs, bx, gamma, &SL, &SR, &cfL, &cfR);
  *sL_out = SL;
  *sR_out = SR;
  const R EL = total_energy(L, bx, gamma), ER = total_energy(Rs, bx, gamma);
  R FL[7], FR[7], UL[7], UR[7];
  physical_flux(L, bx, EL, FL);
  physical_flux(Rs, bx, ER, FR);
  if (SL > R(0.0)) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q];
    return;
  }
  if (SR < R(0.0)) {
    for (int q = 0; q < 7; ++q) F[q] = FR[q];
    return;
  }
  cons_vec(L, EL, UL);
  cons_vec(Rs, ER, UR);
  for (int q = 0; q < 7; ++q)
    F[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) / (SR - SL);
}

// Riemann solver selected by code: 1 Rusanov, 2 HLL, 4 HLLD.
template <class R>
void riemann(int solver, const State<R>& L, const State<R>& Rs, R bx, double gamma, R F[7],
             R* sL, R* sR) {
  if (solver == 1) rusanov(L, Rs, bx, gamma, F, sL, sR);
  else if (solver == 2) hll(L, Rs, bx, gamma, F, sL, sR);
  else hlld(L, Rs, bx, gamma, F, sL, sR);
}

// ---------------------------------------------------------------------------
// E^c edge EMF (Gardiner & Stone 2005), default scheme of Sec. 2.4.
// Generic edge along e with first direction a and second direction b.
// The derivative of the EMF along b, taken on an a-face, is upwinded in a by the
// sign of that a-face's mass flux (averaged when it is exactly zero); likewise
// the derivative along a on a b-face is upwinded in b.
// ---------------------------------------------------------------------------
template <class R>
R emf_ec(const R X[2], const R Y[2], const R C[2][2], const R Fa[2], const R Fb[2], R da, R db) {
  // index 0 = upper (J or I), index 1 = lower (J-1 or I-1)
  R dB_q1, dB_q3, dA_q1, dA_q3;
  {
    // d/db at J-1/4: 2 (C(c, J) - Y(c)) / db, column c chosen by Fa(J)
    const R up = R(2.0) * (C[1][0] - Y[1]) / db;  // column I-1 (upwind for Fa > 0)
    const R dn = R(2.0) * (C[0][0] - Y[0]) / db;  // column I
    if (Fa[0] > R(0.0)) dB_q1 = up;
    else if (Fa[0] < R(0.0)) dB_q1 = dn;
    else dB_q1 = R(0.5) * (up + dn);
  }
  {
    // d/db at J-3/4: 2 (Y(c) - C(c, J-1)) / db, column c chosen by Fa(J-1)
    const R up = R(2.0) * (Y[1] - C[1][1]) / db;
    const R dn = R(2.0) * (Y[0] - C[0][1]) / db;
    if (Fa[1] > R(0.0)) dB_q3 = up;
    else if (Fa[1] < R(0.0)) dB_q3 = dn;
    else dB_q3 = R(0.5) * (up + dn);
  }
  {
    // d/da at I-1/4: 2 (C(I, r) - X(r)) / da, row r chosen by Fb(I)
    const R up = R(2.0) * (C[0][1] - X[1]) / da;  // row J-1 (upwind for Fb > 0)
    const R dn = R(2.0) * (C[0][0] - X[0]) / da;  // row J
    if (Fb[0] > R(0.0)) dA_q1 = up;
    else if (Fb[0] < R(0.0)) dA_q1 = dn;
    else dA_q1 = R(0.5) * (up + dn);
  }
  {
    // d/da at I-3/4: 2 (X(r) - C(I-1, r)) / da, row r chosen by Fb(I-1)
    const R up = R(2.0) * (X[1] - C[1][1]) / da;
    const R dn = R(2.0) * (X[0] - C[1][0]) / da;
    if (Fb[1] > R(0.0)) dA_q3 = up;
    else if (Fb[1] < R(0.0)) dA_q3 = dn;
    else dA_q3 = R(0.5) * (up + dn);
  }
  return R(0.25) * (X[0] + X[1] + Y[0] + Y[1]) + (db / R(8.0)) * (dB_q3 - dB_q1) +
         (da / R(8.0)) * (dA_q3 - dA_q1);
}

// ---------------------------------------------------------------------------
// Face states and fluxes for one direction d.  The face "p" of direction d is
// the face on the lower side of cell p.  Flux storage per direction: 8 slots in
// the global conserved ordering (slot 5 + d, the normal field, stays 0), plus
// the face signal speed max(|S_L|, |S_R|).
// ---------------------------------------------------------------------------
// recon: 1 PLM with the van Leer limiter, 3 LimO3 (both Sec. 2.3)
template <class R>
void face_state(const Grid& G, const std::vector<R>* W, int i, int j, int k, int d, int side,
                State<R>* s, int recon = 1) {
  // side = -1: "left" state of face p, i.e. the +1/2 extrapolation of cell p - e_d
  // side = +1: "right" state of face p, the -1/2 extrapolation of cell p
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  const int c0 = (side < 0) ? -1 : 0;  // the cell being extrapolated, relative to p
  const long pm = shift(G, i, j, k, d, c0 - 1);
  const long p0 = shift(G, i, j, k, d, c0);
  const long pp = shift(G, i, j, k, d, c0 + 1);
  const int var[7] = {RHO, 1 + d, 1 + t1, 1 + t2, PR, 5 + t1, 5 + t2};
  R out[7];
  for (int q = 0; q < 7; ++q) {
    const std::vector<R>& f = W[var[q]];
    if (recon == 3) {
      in_part<R>(ORA_PART_FACE);
      out[q] = (side < 0) ? limo3_face(f[pm], f[p0], f[pp]) : limo3_face(f[pp], f[p0], f[pm]);
      continue;
    }
    in_part<R>(ORA_PART_SLOPE);
    const R slope = vanleer(f[pm], f[p0], f[pp]);
    in_part<R>(ORA_PART_FACE);
    out[q] = (side < 0) ? f[p0] + R(0.5) * slope : f[p0] - R(0.5) * slope;
  }
  s->rho = out[0]; s->u = out[1]; s->v = out[2]; s->w = out[3]; s->P = out[4];
  s->by = out[5]; s->bz = out[6];
}

template <class R>
void face_fluxes(const Grid& G, double gamma, const std::vector<R>* U, const std::vector<R>* W,
                 int d, std::vector<R>* F /*8*/, std::vector<R>& cface, int solver,
                 int recon = 1) {
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
#pragma omp parallel for if (kPar<R>)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        State<R> L, Rr;
        face_state(G, W, i, j, k, d, -1, &L, recon);
        face_state(G, W, i, j, k, d, +1, &Rr, recon);
        const R bn = U[5 + d][p];
        R f[7], sL, sR;
        in_part<R>(ORA_PART_RIEMANN);
        riemann(solver, L, Rr, bn, gamma, f, &sL, &sR);
        F[RHO][p] = f[0];
        F[1 + d][p] = f[1];
        F[1 + t1][p] = f[2];
        F[1 + t2][p] = f[3];
        F[EN][p] = f[4];
        F[5 + d][p] = R(0.0);
        F[5 + t1][p] = f[5];
        F[5 + t2][p] = f[6];
        in_part<R>(ORA_PART_SPEED);
        cface[p] = rmax(absval(sL), absval(sR));
      }
}

template <class R>
void face_speeds(const Grid& G, double gamma, const std::vector<R>* U, const std::vector<R>* W,
                 int d, std::vector<R>& cface, int recon = 1) {
#pragma omp parallel for if (kPar<R>)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        State<R> L, Rr;
        face_state(G, W, i, j, k, d, -1, &L, recon);
        face_state(G, W, i, j, k, d, +1, &Rr, recon);
        const R bn = U[5 + d][p];
        const R cfL = fast_speed(L, bn, gamma);
        const R cfR = fast_speed(Rr, bn, gamma);
        const R cfmax = rmax(cfL, cfR);
        const R sL = rmin(L.u, Rr.u) - cfmax;
        const R sR = rmax(L.u, Rr.u) + cfmax;
        cface[p] = rmax(absval(sL), absval(sR));
      }
}

// Inverse CFL time of Eq. (10) with no diffusion: max over cells of
// sum over integrated directions of max(c at the two faces) / dl.
template <class R> R inverse_dt(const Grid& G, const std::vector<R>* cface) {
  in_part<R>(ORA_PART_INVDT);
  std::vector<R> plane_max(G.n[2], R(0.0));
#pragma omp parallel for if (kPar<R>)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        R s = R(0.0);
        for (int d = 0; d < 3; ++d) {
          if (!G.active[d]) continue;
          const R c = rmax(cface[d][p], cface[d][shift(G, i, j, k, d, 1)]);
          s = s + c / R(G.dl[d]);
        }
        plane_max[k] = rmax(plane_max[k], s);
      }
  R best = R(0.0);
  for (int k = 0; k < G.n[2]; ++k) best = rmax(best, plane_max[k]);
  return best;
}

// EMF component e at every edge (stored at the cell whose lower a- and b-faces
// bound the edge), with a = e+1, b = e+2 (mod 3).
template <class R>
void edge_emf(const Grid& G, const std::vector<R>* W, const std::vector<R>* F /*[3][8]*/, int e,
              std::vector<R>& Ee) {
  const int a = (e + 1) % 3, b = (e + 2) % 3;
#pragma omp parallel for if (kPar<R>)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        R X[2], Y[2], C[2][2], Fa[2], Fb[2];
        for (int r = 0; r < 2; ++r) {
          // a-face at p - r e_b: EMF_e = -F_a[B_b]
          const long q = shift(G, i, j, k, b, -r);
          X[r] = -F[8 * a + 5 + b][q];
          Fa[r] = F[8 * a + RHO][q];
        }
        for (int c = 0; c < 2; ++c) {
          // b-face at p - c e_a: EMF_e = +F_b[B_a]
          const long q = shift(G, i, j, k, a, -c);
          Y[c] = F[8 * b + 5 + a][q];
          Fb[c] = F[8 * b + RHO][q];
        }
        in_part<R>(ORA_PART_CELL_EMF);
        for (int c = 0; c < 2; ++c)
          for (int r = 0; r < 2; ++r) {
            // cell-centre EMF_e = -(v x B)_e = -(v_a B_b - v_b B_a)
            const long q = shift2(G, i, j, k, a, -c, b, -r);
            C[c][r] = -(W[1 + a][q] * W[5 + b][q] - W[1 + b][q] * W[5 + a][q]);
          }
        in_part<R>(ORA_PART_EDGE);
        Ee[at(G, i, j, k)] = emf_ec(X, Y, C, Fa, Fb, R(G.dl[a]), R(G.dl[b]));
      }
}

// ---------------------------------------------------------------------------
// Vector-potential form of the induction equation (Sec. 2.4, Eqs. 7-8): A lives on
// the cell edges where the EMF lives, dA/dt = -E there, and every face field is the
// circulation of A around that face divided by its area (Stokes), B = curl A.  A_e is
// stored like E_e: at the cell whose lower a- and b-faces bound the edge.  The face
// field is Bref + curl A, Bref a fixed face field: a uniform mean field (which a
// periodic A cannot represent), or the field a run started from with A = 0 there
// (the gauge A = -integral of E dt from that moment).
// A difference along a direction with one cell vanishes, so that term is dropped.
// ---------------------------------------------------------------------------
template <class R>
void curl_faces(const Grid& G, const std::vector<R>* A, const std::vector<R>* Bref,
                std::vector<R>* B) {
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        for (int d = 0; d < 3; ++d) {
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          R b = Bref[d][p];
          if (G.active[t1]) b = b + (A[t2][shift(G, i, j, k, t1, 1)] - A[t2][p]) / R(G.dl[t1]);
          if (G.active[t2]) b = b - (A[t1][shift(G, i, j, k, t2, 1)] - A[t1][p]) / R(G.dl[t2]);
          B[d][p] = b;
        }
      }
}

// The EMF that drives A_e in a stage.  Both transverse directions a = e+1, b = e+2
// integrated: the E^c edge EMF.  Only a integrated: the edge collapses onto the a-face
// of the cell and E_e = -F_a[B_b] there; only b integrated: E_e = +F_b[B_a] on the
// b-face (E = -v x B, and F_a[B_b] = v_a B_b - v_b B_a).  The curl of these is the
// divergence of the face fluxes of the field normal to the thin direction, as in the
// field form.  Neither integrated: A_e enters no face field; its EMF is taken as 0.
template <class R>
void potential_emf(const Grid& G, const std::vector<R>* W, const std::vector<R>* F /*[3][8]*/,
                   int e, std::vector<R>& Ee) {
  const int a = (e + 1) % 3, b = (e + 2) % 3;
  if (G.active[a] && G.active[b]) {
    edge_emf(G, W, F, e, Ee);
  } else if (G.active[a]) {
    for (long p = 0; p < G.ncell; ++p) Ee[p] = -F[8 * a + 5 + b][p];
  } else if (G.active[b]) {
    for (long p = 0; p < G.ncell; ++p) Ee[p] = F[8 * b + 5 + a][p];
  } else {
    for (long p = 0; p < G.ncell; ++p) Ee[p] = R(0.0);
  }
}

// ---------------------------------------------------------------------------
// One stage of Sec. 2.7: U* = S_dt(Uin), Uout = w U* + w0 U0 (Eq. 9).
// ---------------------------------------------------------------------------
template <class R>
int stage(const Grid& G, double gamma, R dt, const std::vector<R>* Uin, const std::vector<R>* U0,
          double w, double w0, std::vector<R>* Uout, R* inv_dt, long* bad, int solver = 4,
          const std::vector<R>* Ain = nullptr, const std::vector<R>* A0 = nullptr,
          std::vector<R>* Aout = nullptr, const std::vector<R>* Bref = nullptr, int recon = 1) {
  const long N = G.ncell;
  std::vector<R> W[8];
  for (int f = 0; f < 8; ++f) W[f].assign(N, R(0.0));
  int st = prims(G, gamma, Uin, W, bad);
  if (st != ORA_OK) return st;

  std::vector<R> F[24];  // F[8 * d + slot]
  std::vector<R> cface[3];
  for (int q = 0; q < 24; ++q) F[q].assign(N, R(0.0));
  for (int d = 0; d < 3; ++d) {
    cface[d].assign(N, R(0.0));
    if (G.active[d]) face_fluxes(G, gamma, Uin, W, d, &F[8 * d], cface[d], solver, recon);
  }
  *inv_dt = inverse_dt(G, cface);

  // EMF along e is needed only when both other directions are integrated.
  std::vector<R> Eedge[3];
  for (int e = 0; e < 3; ++e) {
    Eedge[e].assign(N, R(0.0));
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    if (G.active[a] && G.active[b]) edge_emf(G, W, F, e, Eedge[e]);
  }

  std::vector<R> Us[8];
  for (int f = 0; f < 8; ++f) Us[f].assign(N, R(0.0));
#pragma omp parallel for if (kPar<R>)
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        // cell-averaged conserved variables: U* = U - dt sum_d dF_d / dl_d
        for (int f = 0; f < 5; ++f) {
          in_part<R>(ORA_PART_DIFF);
          R div = R(0.0);
          for (int d = 0; d < 3; ++d) {
            if (!G.active[d]) continue;
            div = div + (F[8 * d + f][shift(G, i, j, k, d, 1)] - F[8 * d + f][p]) / R(G.dl[d]);
          }
          in_part<R>(ORA_PART_ACCUM);
          Us[f][p] = Uin[f][p] - dt * div;
        }
        // face-centred field: B_d* = B_d - dt (curl E)_d (Eq. 6, Stokes on the face)
        for (int d = 0; d < 3; ++d) {
          const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
          in_part<R>(ORA_PART_DIFF);
          R curl = R(0.0);
          if (G.active[d]) {
            if (G.active[t1])
              curl = curl + (Eedge[t2][shift(G, i, j, k, t1, 1)] - Eedge[t2][p]) / R(G.dl[t1]);
            if (G.active[t2])
              curl = curl - (Eedge[t1][shift(G, i, j, k, t2, 1)] - Eedge[t1][p]) / R(G.dl[t2]);
          } else {
            // B_d along a non-integrated direction is cell-like in d: the exact
            // reduction of the CT update is the divergence of the face fluxes of B_d.
            for (int a = 0; a < 3; ++a) {
              if (a == d || !G.active[a]) continue;
              curl = curl + (F[8 * a + 5 + d][shift(G, i, j, k, a, 1)] - F[8 * a + 5 + d][p]) /
                                R(G.dl[a]);
            }
          }
          in_part<R>(ORA_PART_ACCUM);
          Us[5 + d][p] = Uin[5 + d][p] - dt * curl;
        }
      }

  in_part<R>(ORA_PART_COMBINE);
  for (int f = 0; f < 8; ++f)
    for (long p = 0; p < N; ++p) {
      if (w0 == 0.0 && w == 1.0)
        Uout[f][p] = Us[f][p];
      else
        Uout[f][p] = R(w) * Us[f][p] + R(w0) * U0[f][p];
    }
  if (Ain == nullptr) return ORA_OK;
  in_part<R>(ORA_PART_POTENTIAL);

  // Vector-potential form (Eqs. 7-8): A* = A - dt E, A_out = w A* + w0 A_0, and the
  // face field is recomputed from A_out instead of being stepped itself.
  for (int e = 0; e < 3; ++e) {
    std::vector<R> Ee(N, R(0.0));
    potential_emf(G, W, F, e, Ee);
    for (long p = 0; p < N; ++p) {
      const R As = Ain[e][p] - dt * Ee[p];
      Aout[e][p] = (w0 == 0.0 && w == 1.0) ? As : R(w) * As + R(w0) * A0[e][p];
    }
  }
  curl_faces(G, Aout, Bref, &Uout[5]);
  return ORA_OK;
}

// One RK cycle of Sec. 2.7, same dt for every stage, stage s: U_s = w_s S_dt(U_{s-1}) +
// w0_s U_0 with the weights of Table 1 -- RK2: (1, 0), (1/2, 1/2); RK3: (1, 0),
// (1/4, 3/4), (2/3, 1/3).  The next dt comes from the largest inverse CFL time of the
// cycle's stages.
template <class R>
int cycle(const Grid& G, double gamma, double cfl, std::vector<R>* U, R* inv_dt, double dt_max,
          R* dt_taken, long* bad, int solver = 4, int rk_order = 2, std::vector<R>* A = nullptr,
          const std::vector<R>* Bref = nullptr, int recon = 1) {
  in_part<R>(ORA_PART_DT);
  R dt = R(cfl) / *inv_dt;
  if (value(dt) > dt_max) dt = R(dt_max);
  const long N = G.ncell;
  const double w_rk2[2][2] = {{1.0, 0.0}, {0.5, 0.5}};
  const double w_rk3[3][2] = {{1.0, 0.0}, {0.25, 0.75}, {2.0 / 3.0, 1.0 / 3.0}};
  const int nst = rk_order == 3 ? 3 : 2;
  std::vector<R> prev[8], next[8], prevA[3], nextA[3];
  for (int f = 0; f < 8; ++f) prev[f] = U[f];
  if (A)
    for (int e = 0; e < 3; ++e) prevA[e] = A[e];
  R inv = R(0.0);
  for (int st = 0; st < nst; ++st) {
    const double w = rk_order == 3 ? w_rk3[st][0] : w_rk2[st][0];
    const double w0 = rk_order == 3 ? w_rk3[st][1] : w_rk2[st][1];
    for (int f = 0; f < 8; ++f) next[f].assign(N, R(0.0));
    if (A)
      for (int e = 0; e < 3; ++e) nextA[e].assign(N, R(0.0));
    R inv_s;
    const int rc = stage(G, gamma, dt, prev, st == 0 ? (const std::vector<R>*)nullptr : U, w, w0,
                         next, &inv_s, bad, solver, A ? prevA : nullptr,
                         (A && st > 0) ? A : nullptr, A ? nextA : nullptr, Bref, recon);
    if (rc != ORA_OK) return rc;
    in_part<R>(ORA_PART_DT);
    inv = rmax(inv, inv_s);
    for (int f = 0; f < 8; ++f) prev[f].swap(next[f]);
    if (A)
      for (int e = 0; e < 3; ++e) prevA[e].swap(nextA[e]);
  }
  for (int f = 0; f < 8; ++f) U[f] = prev[f];
  if (A)
    for (int e = 0; e < 3; ++e) A[e] = prevA[e];
  *inv_dt = inv;
  *dt_taken = dt;
  return ORA_OK;
}

// ---- marshalling helpers -------------------------------------------------
void load(const Grid& G, const double* const src[8], std::vector<double>* dst) {
  for (int f = 0; f < 8; ++f) dst[f].assign(src[f], src[f] + G.ncell);
}
void store(const Grid& G, const std::vector<double>* src, double* const dst[8]) {
  for (int f = 0; f < 8; ++f) std::memcpy(dst[f], src[f].data(), sizeof(double) * G.ncell);
}
bool ptrs_ok(const void* const p[8]) {
  if (!p) return false;
  for (int f = 0; f < 8; ++f)
    if (!p[f]) return false;
  return true;
}

}  // namespace

// ===========================================================================
// C interface
// ===========================================================================
extern "C" {

int ora_cons_from_prims(const ora_grid* g, double gamma, const double* const prim[8],
                        double* const cons[8]) {
  if (!grid_ok(g) || !(gamma > 1.0) || !ptrs_ok((const void* const*)prim) ||
      !ptrs_ok((const void* const*)cons))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> out[8];
  for (int f = 0; f < 8; ++f) out[f].assign(G.ncell, 0.0);
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        const long p = at(G, i, j, k);
        const double rho = prim[0][p], vx = prim[1][p], vy = prim[2][p], vz = prim[3][p];
        const double P = prim[4][p];
        const double bx = 0.5 * (prim[5][p] + prim[5][shift(G, i, j, k, 0, 1)]);
        const double by = 0.5 * (prim[6][p] + prim[6][shift(G, i, j, k, 1, 1)]);
        const double bz = 0.5 * (prim[7][p] + prim[7][shift(G, i, j, k, 2, 1)]);
        out[RHO][p] = rho;
        out[MX][p] = rho * vx;
        out[MY][p] = rho * vy;
        out[MZ][p] = rho * vz;
        out[EN][p] = P / (gamma - 1.0) + 0.5 * rho * (vx * vx + vy * vy + vz * vz) +
                     0.5 * (bx * bx + by * by + bz * bz);
        out[BX][p] = prim[5][p];
        out[BY][p] = prim[6][p];
        out[BZ][p] = prim[7][p];
      }
  store(G, out, cons);
  return ORA_OK;
}

int ora_prims(const ora_grid* g, double gamma, const double* const cons[8], double* const w[8],
              long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !ptrs_ok((const void* const*)cons) ||
      !ptrs_ok((const void* const*)w))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8], W[8];
  load(G, cons, U);
  for (int f = 0; f < 8; ++f) W[f].assign(G.ncell, 0.0);
  const int st = prims(G, gamma, U, W, bad_cell);
  store(G, W, w);
  return st;
}

double ora_vanleer(double wm, double w0, double wp) { return vanleer<double>(wm, w0, wp); }

int ora_hlld(const double wL[7], const double wR[7], double bn, double gamma, double F[7],
             double* sL, double* sR) {
  if (!wL || !wR || !F || !sL || !sR || !(gamma > 1.0)) return ORA_EINVAL;
  State<double> L{wL[0], wL[1], wL[2], wL[3], wL[4], wL[5], wL[6]};
  State<double> R{wR[0], wR[1], wR[2], wR[3], wR[4], wR[5], wR[6]};
  if (!(L.rho > 0) || !(R.rho > 0) || !(L.P > 0) || !(R.P > 0)) return ORA_ENONPHYS;
  hlld(L, R, bn, gamma, F, sL, sR);
  return ORA_OK;
}

int ora_phys_flux(const double w[7], double bn, double gamma, double F[7]) {
  if (!w || !F || !(gamma > 1.0)) return ORA_EINVAL;
  State<double> s{w[0], w[1], w[2], w[3], w[4], w[5], w[6]};
  physical_flux(s, bn, total_energy(s, bn, gamma), F);
  return ORA_OK;
}

double ora_emf_ec(const double X[2], const double Y[2], const double C[2][2], const double Fa[2],
                  const double Fb[2], double da, double db) {
  return emf_ec<double>(X, Y, C, Fa, Fb, da, db);
}

int ora_speed_pass(const ora_grid* g, double gamma, const double* const cons[8], double* inv_dt,
                   long* bad_cell) {
  return ora_speed_pass_recon(g, gamma, 1, cons, inv_dt, bad_cell);
}

double ora_limo3_face(double w_back, double w0, double w_face) {
  return limo3_face<double>(w_back, w0, w_face);
}

int ora_speed_pass_recon(const ora_grid* g, double gamma, int recon, const double* const cons[8],
                         double* inv_dt, long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !ptrs_ok((const void* const*)cons) || !inv_dt ||
      (recon != 1 && recon != 3))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8], W[8], cface[3];
  load(G, cons, U);
  for (int f = 0; f < 8; ++f) W[f].assign(G.ncell, 0.0);
  const int st = prims(G, gamma, U, W, bad_cell);
  if (st != ORA_OK) return st;
  for (int d = 0; d < 3; ++d) {
    cface[d].assign(G.ncell, 0.0);
    if (G.active[d]) face_speeds(G, gamma, U, W, d, cface[d], recon);
  }
  *inv_dt = inverse_dt(G, cface);
  return ORA_OK;
}

int ora_stage(const ora_grid* g, double gamma, double dt, const double* const uin[8],
              const double* const u0[8], double w, double w0, double* const uout[8],
              double* inv_dt, long* bad_cell) {
  return ora_stage_scheme(g, gamma, dt, 1, 4, uin, u0, w, w0, uout, inv_dt, bad_cell);
}

int ora_stage_scheme(const ora_grid* g, double gamma, double dt, int recon, int solver,
                     const double* const uin[8], const double* const u0[8], double w, double w0,
                     double* const uout[8], double* inv_dt, long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !ptrs_ok((const void* const*)uin) ||
      !ptrs_ok((const void* const*)uout) || !inv_dt || !(dt >= 0.0) ||
      (recon != 1 && recon != 3) || (solver != 1 && solver != 2 && solver != 4))
    return ORA_EINVAL;
  if (w0 != 0.0 && !ptrs_ok((const void* const*)u0)) return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> Ui[8], U0[8], Uo[8];
  load(G, uin, Ui);
  if (w0 != 0.0) load(G, u0, U0);
  for (int f = 0; f < 8; ++f) Uo[f].assign(G.ncell, 0.0);
  double inv = 0.0;
  const int st = stage<double>(G, gamma, dt, Ui, U0, w, w0, Uo, &inv, bad_cell, solver, nullptr,
                               nullptr, nullptr, nullptr, recon);
  if (st != ORA_OK) return st;
  store(G, Uo, uout);
  *inv_dt = inv;
  return ORA_OK;
}

int ora_cycle(const ora_grid* g, double gamma, double cfl, double* const u[8], double* inv_dt,
              double dt_max, double* dt_taken, long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !(cfl > 0.0 && cfl < 1.0) ||
      !ptrs_ok((const void* const*)u) || !inv_dt || !(*inv_dt > 0.0) || !(dt_max >= 0.0))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8];
  load(G, (const double* const*)u, U);
  double inv = *inv_dt, dt = 0.0;
  const int st = cycle(G, gamma, cfl, U, &inv, dt_max, &dt, bad_cell);
  if (st != ORA_OK) return st;
  store(G, U, u);
  *inv_dt = inv;
  if (dt_taken) *dt_taken = dt;
  return ORA_OK;
}

int ora_riemann(int solver, const double wL[7], const double wR[7], double bn, double gamma,
                double F[7], double* sL, double* sR) {
  if (!wL || !wR || !F || !sL || !sR || !(gamma > 1.0)) return ORA_EINVAL;
  if (solver != 1 && solver != 2 && solver != 4) return ORA_EINVAL;
  State<double> L{wL[0], wL[1], wL[2], wL[3], wL[4], wL[5], wL[6]};
  State<double> R{wR[0], wR[1], wR[2], wR[3], wR[4], wR[5], wR[6]};
  if (!(L.rho > 0) || !(R.rho > 0) || !(L.P > 0) || !(R.P > 0)) return ORA_ENONPHYS;
  riemann(solver, L, R, bn, gamma, F, sL, sR);
  return ORA_OK;
}

int ora_cycle_rk(const ora_grid* g, double gamma, double cfl, int solver, int rk_order,
                 double* const u[8], double* inv_dt, double dt_max, double* dt_taken,
                 long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !(cfl > 0.0 && cfl < 1.0) ||
      !ptrs_ok((const void* const*)u) || !inv_dt || !(*inv_dt > 0.0) || !(dt_max >= 0.0))
    return ORA_EINVAL;
  if ((solver != 1 && solver != 2 && solver != 4) || (rk_order != 2 && rk_order != 3))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8];
  load(G, (const double* const*)u, U);
  double inv = *inv_dt, dt = 0.0;
  const int st = cycle(G, gamma, cfl, U, &inv, dt_max, &dt, bad_cell, solver, rk_order);
  if (st != ORA_OK) return st;
  store(G, U, u);
  *inv_dt = inv;
  if (dt_taken) *dt_taken = dt;
  return ORA_OK;
}

int ora_cycle_solver(const ora_grid* g, double gamma, double cfl, int solver, double* const u[8],
                     double* inv_dt, double dt_max, double* dt_taken, long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !(cfl > 0.0 && cfl < 1.0) ||
      !ptrs_ok((const void* const*)u) || !inv_dt || !(*inv_dt > 0.0) || !(dt_max >= 0.0))
    return ORA_EINVAL;
  if (solver != 1 && solver != 2 && solver != 4) return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8];
  load(G, (const double* const*)u, U);
  double inv = *inv_dt, dt = 0.0;
  const int st = cycle(G, gamma, cfl, U, &inv, dt_max, &dt, bad_cell, solver);
  if (st != ORA_OK) return st;
  store(G, U, u);
  *inv_dt = inv;
  if (dt_taken) *dt_taken = dt;
  return ORA_OK;
}

int ora_b_from_potential(const ora_grid* g, const double* const A[3], const double bmean[3],
                         double* const B[3]) {
  if (!grid_ok(g) || !A || !bmean || !B) return ORA_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!A[d] || !B[d]) return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> Av[3], Bref[3], Bv[3];
  for (int d = 0; d < 3; ++d) {
    Av[d].assign(A[d], A[d] + G.ncell);
    Bref[d].assign(G.ncell, bmean[d]);
    Bv[d].assign(G.ncell, 0.0);
  }
  curl_faces(G, Av, Bref, Bv);
  for (int d = 0; d < 3; ++d) std::memcpy(B[d], Bv[d].data(), sizeof(double) * G.ncell);
  return ORA_OK;
}

int ora_cycle_vp(const ora_grid* g, double gamma, double cfl, int solver, int rk_order,
                 double* const u[8], double* const A[3], const double* const Bref[3],
                 double* inv_dt, double dt_max, double* dt_taken, long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !(cfl > 0.0 && cfl < 1.0) ||
      !ptrs_ok((const void* const*)u) || !inv_dt || !(*inv_dt > 0.0) || !(dt_max >= 0.0) ||
      !A || !Bref)
    return ORA_EINVAL;
  for (int e = 0; e < 3; ++e)
    if (!A[e] || !Bref[e]) return ORA_EINVAL;
  if ((solver != 1 && solver != 2 && solver != 4) || (rk_order != 2 && rk_order != 3))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8], Av[3], Br[3];
  load(G, (const double* const*)u, U);
  for (int e = 0; e < 3; ++e) {
    Av[e].assign(A[e], A[e] + G.ncell);
    Br[e].assign(Bref[e], Bref[e] + G.ncell);
  }
  double inv = *inv_dt, dt = 0.0;
  const int st = cycle(G, gamma, cfl, U, &inv, dt_max, &dt, bad_cell, solver, rk_order, Av, Br);
  if (st != ORA_OK) return st;
  store(G, U, u);
  for (int e = 0; e < 3; ++e) std::memcpy(A[e], Av[e].data(), sizeof(double) * G.ncell);
  *inv_dt = inv;
  if (dt_taken) *dt_taken = dt;
  return ORA_OK;
}

int ora_cycle_scheme(const ora_grid* g, double gamma, double cfl, int recon, int solver,
                     int rk_order, double* const u[8], double* const A[3],
                     const double* const Bref[3], double* inv_dt, double dt_max,
                     double* dt_taken, long* bad_cell) {
  if (!grid_ok(g) || !(gamma > 1.0) || !(cfl > 0.0 && cfl < 1.0) ||
      !ptrs_ok((const void* const*)u) || !inv_dt || !(*inv_dt > 0.0) || !(dt_max >= 0.0))
    return ORA_EINVAL;
  if ((recon != 1 && recon != 3) || (solver != 1 && solver != 2 && solver != 4) ||
      (rk_order != 2 && rk_order != 3) || (!A) != (!Bref))
    return ORA_EINVAL;
  if (A)
    for (int e = 0; e < 3; ++e)
      if (!A[e] || !Bref[e]) return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8], Av[3], Br[3];
  load(G, (const double* const*)u, U);
  if (A)
    for (int e = 0; e < 3; ++e) {
      Av[e].assign(A[e], A[e] + G.ncell);
      Br[e].assign(Bref[e], Bref[e] + G.ncell);
    }
  double inv = *inv_dt, dt = 0.0;
  const int st = cycle(G, gamma, cfl, U, &inv, dt_max, &dt, bad_cell, solver, rk_order,
                       A ? Av : nullptr, A ? Br : nullptr, recon);
  if (st != ORA_OK) return st;
  store(G, U, u);
  if (A)
    for (int e = 0; e < 3; ++e) std::memcpy(A[e], Av[e].data(), sizeof(double) * G.ncell);
  *inv_dt = inv;
  if (dt_taken) *dt_taken = dt;
  return ORA_OK;
}

int ora_count_cycle_parts(const ora_grid* g, double gamma, double cfl, const double* const u[8],
                          double inv_dt, double counts[5 * ORA_NUM_PARTS]) {
  if (!grid_ok(g) || !(gamma > 1.0) || !ptrs_ok((const void* const*)u) || !counts ||
      !(inv_dt > 0.0))
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<Counted> U[8];
  for (int f = 0; f < 8; ++f) {
    U[f].resize(G.ncell);
    for (long p = 0; p < G.ncell; ++p) U[f][p] = Counted(u[f][p]);
  }
  reset_tally();
  Counted inv(inv_dt), dt;
  long bad = -1;
  const int st =
      cycle(G, gamma, cfl, U, &inv, std::numeric_limits<double>::infinity(), &dt, &bad);
  const double n = (double)G.ncell;
  for (int q = 0; q < ORA_NUM_PARTS; ++q) {
    counts[5 * q + 0] = g_parts[q].add / n;
    counts[5 * q + 1] = g_parts[q].mul / n;
    counts[5 * q + 2] = g_parts[q].div / n;
    counts[5 * q + 3] = g_parts[q].sqrt / n;
    counts[5 * q + 4] = g_parts[q].cmp / n;
  }
  reset_tally();
  return st;
}

int ora_count_cycle(const ora_grid* g, double gamma, double cfl, const double* const u[8],
                    double inv_dt, double counts[5]) {
  if (!counts) return ORA_EINVAL;
  double parts[5 * ORA_NUM_PARTS];
  const int st = ora_count_cycle_parts(g, gamma, cfl, u, inv_dt, parts);
  if (st == ORA_EINVAL) return st;
  for (int k = 0; k < 5; ++k) {
    counts[k] = 0.0;
    for (int q = 0; q < ORA_NUM_PARTS; ++q) counts[k] += parts[5 * q + k];
  }
  return st;
}

namespace {
// The tally of everything counted since the last reset, into counts[5].
void total_tally(double counts[5]) {
  for (int k = 0; k < 5; ++k) counts[k] = 0.0;
  for (int q = 0; q < ORA_NUM_PARTS; ++q) {
    counts[0] += g_parts[q].add; counts[1] += g_parts[q].mul; counts[2] += g_parts[q].div;
    counts[3] += g_parts[q].sqrt; counts[4] += g_parts[q].cmp;
  }
}
State<Counted> counted_state(const double w[7]) {
  return State<Counted>{w[0], w[1], w[2], w[3], w[4], w[5], w[6]};
}
}  // namespace

int ora_count_vanleer(double wm, double w0, double wp, double counts[5]) {
  if (!counts) return ORA_EINVAL;
  reset_tally();
  vanleer<Counted>(wm, w0, wp);
  total_tally(counts);
  reset_tally();
  return ORA_OK;
}

int ora_count_energy_flux(const double w[7], double bn, double gamma, double counts_energy[5],
                          double counts_flux[5]) {
  if (!w || !counts_energy || !counts_flux || !(gamma > 1.0)) return ORA_EINVAL;
  const State<Counted> s = counted_state(w);
  reset_tally();
  const Counted E = total_energy(s, Counted(bn), gamma);
  total_tally(counts_energy);
  reset_tally();
  Counted F[7];
  physical_flux(s, Counted(bn), Counted(value(E)), F);
  total_tally(counts_flux);
  reset_tally();
  return ORA_OK;
}

int ora_count_hlld(const double wL[7], const double wR[7], double bn, double gamma,
                   double counts[5]) {
  if (!wL || !wR || !counts || !(gamma > 1.0)) return ORA_EINVAL;
  if (!(wL[0] > 0) || !(wR[0] > 0) || !(wL[4] > 0) || !(wR[4] > 0)) return ORA_ENONPHYS;
  const State<Counted> L = counted_state(wL), R = counted_state(wR);
  reset_tally();
  Counted F[7], sL, sR;
  hlld(L, R, Counted(bn), gamma, F, &sL, &sR);
  total_tally(counts);
  reset_tally();
  return ORA_OK;
}

int ora_count_emf_ec(const double X[2], const double Y[2], const double C[2][2],
                     const double Fa[2], const double Fb[2], double da, double db,
                     double counts[5]) {
  if (!X || !Y || !C || !Fa || !Fb || !counts) return ORA_EINVAL;
  const Counted Xc[2] = {X[0], X[1]}, Yc[2] = {Y[0], Y[1]};
  const Counted Cc[2][2] = {{C[0][0], C[0][1]}, {C[1][0], C[1][1]}};
  const Counted Fac[2] = {Fa[0], Fa[1]}, Fbc[2] = {Fb[0], Fb[1]};
  reset_tally();
  emf_ec<Counted>(Xc, Yc, Cc, Fac, Fbc, Counted(da), Counted(db));
  total_tally(counts);
  reset_tally();
  return ORA_OK;
}

}  // extern "C"

namespace {
// Per-face counts of direction d: the HLLD solve, the reconstruction of both face states,
// and (split, nullable) the HLLD solve, the slopes and the face values.
int count_faces_split(const ora_grid* g, double gamma, const double* const u[8], int d,
                      double counts_hlld[5], double counts_recon[5], double* split) {
  if (!grid_ok(g) || !(gamma > 1.0) || !ptrs_ok((const void* const*)u) || d < 0 || d > 2 ||
      !counts_hlld || !counts_recon)
    return ORA_EINVAL;
  const Grid G = make_grid(g);
  std::vector<double> U[8], W[8];
  load(G, u, U);
  for (int f = 0; f < 8; ++f) W[f].assign(G.ncell, 0.0);
  long bad = -1;
  const int st = prims(G, gamma, U, W, &bad);
  if (st != ORA_OK) return st;
  std::vector<Counted> Wc[8];
  for (int f = 0; f < 8; ++f) {
    Wc[f].resize(G.ncell);
    for (long p = 0; p < G.ncell; ++p) Wc[f][p] = Counted(W[f][p]);
  }
  reset_tally();
  for (int k = 0; k < G.n[2]; ++k)
    for (int j = 0; j < G.n[1]; ++j)
      for (int i = 0; i < G.n[0]; ++i) {
        State<Counted> L, R;
        face_state(G, Wc, i, j, k, d, -1, &L);  // tallied under the slope and face parts
        face_state(G, Wc, i, j, k, d, +1, &R);
        in_part<Counted>(ORA_PART_RIEMANN);
        Counted F[7], sL, sR;
        hlld(L, R, Counted(u[5 + d][at(G, i, j, k)]), gamma, F, &sL, &sR);
      }
  Tally riemann = g_parts[ORA_PART_RIEMANN], recon;
  for (int q : {ORA_PART_SLOPE, ORA_PART_FACE}) {
    recon.add += g_parts[q].add; recon.mul += g_parts[q].mul; recon.div += g_parts[q].div;
    recon.sqrt += g_parts[q].sqrt; recon.cmp += g_parts[q].cmp;
  }
  const Tally slope = g_parts[ORA_PART_SLOPE], face = g_parts[ORA_PART_FACE];
  reset_tally();
  const double n = (double)G.ncell;
  const Tally* t[5] = {&riemann, &recon, &riemann, &slope, &face};
  double* out[5] = {counts_hlld, counts_recon, split, split ? split + 5 : nullptr,
                    split ? split + 10 : nullptr};
  for (int q = 0; q < 5; ++q) {
    if (!out[q]) continue;
    out[q][0] = t[q]->add / n; out[q][1] = t[q]->mul / n; out[q][2] = t[q]->div / n;
    out[q][3] = t[q]->sqrt / n; out[q][4] = t[q]->cmp / n;
  }
  return ORA_OK;
}

}  // namespace

extern "C" {

int ora_count_faces_parts(const ora_grid* g, double gamma, const double* const u[8], int d,
                          double counts[15]) {
  if (!counts) return ORA_EINVAL;
  double h[5], r[5];
  return count_faces_split(g, gamma, u, d, h, r, counts);
}

int ora_count_faces(const ora_grid* g, double gamma, const double* const u[8], int d,
                    double counts_hlld[5], double counts_recon[5]) {
  if (!counts_hlld || !counts_recon) return ORA_EINVAL;
  return count_faces_split(g, gamma, u, d, counts_hlld, counts_recon, nullptr);
}

int ora_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
