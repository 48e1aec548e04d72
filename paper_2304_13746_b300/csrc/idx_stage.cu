// idx_stage.cu -- sm_103a kernels of one RK2 cycle of ideal MHD and the C ABI (include/idx.h).
//
// The FP64 stage is bound by the FP64 pipe (1/64 of the FP32 rate on this part), not
// by HBM: it moves ~2.4 KB per cell-update against ~0.5 us of FP64 arithmetic.  So the
// stage is split into kernels that each compute every quantity exactly once --
// primitives per cell, PLM slopes per cell and direction, one HLLD per face, one E^c
// per edge -- and hand their results through HBM, instead of one fused tile kernel
// that would recompute halo faces.  Per stage:
//
//   k_prims      U (8 fields)            -> W: rho, v, P, cell-centre B      (Secs. 2.1, 2.3)
//   k_sweep<d>   W along d, face B_d     -> F_d: 7 HLLD fluxes + face speed  (Sec. 2.3)
//                (one thread marches a pencil segment: slopes computed once per cell)
//   k_emf        F_a, F_b, W             -> edge EMFs E_e (E^c)               (Sec. 2.4)
//   k_update     U, F_d, E_e [, U_0]     -> U_out = w U* + w0 U_0; block max of the
//                                           inverse CFL time -> atomicMax    (Eqs. 5, 6, 9, 10)
//
// A cycle is k_begin (dt from the previous cycle's speeds, clamp to t_end) + 2 stages +
// k_end (t, step count, speeds for the next dt), captured once into a CUDA graph and
// replayed; time, dt and the error flag stay on the device.
//
// FP32 bulk (RK2, field form, periodic) runs k_update_carry in place of k_update: it also
// recovers the primitives of the state it forms, for the next stage, so k_prims drops out
// of the cycle, and it carries the RK2 combine as the half sum (U^n + U*)/2.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <type_traits>
#include <vector>
#include <array>
#include <map>
#include <tuple>

#include "../../include/idx.h"
#include "divmagic.cuh"
#include "mhd_math.cuh"
#include "tma.cuh"

using namespace idx;

namespace {

constexpr int kThreads = 256;
constexpr int kSegDefault = 16;  // faces per thread along a marching sweep, before tuning
constexpr int kTuneMinCells = 1 << 15;  // smaller grids keep the default shapes

// Device control block of one sim.
struct Ctrl {
  double t;
  double t_end;
  double dt;                       // dt of the running cycle; 0 means "skip"
  double cfl;
  double last_dt;                  // dt of the last completed cycle
  unsigned long long inv_prev;     // bits of the inverse CFL time for the next dt
  unsigned long long inv_acc;      // running max (bits) over the current cycle's stages
  unsigned long long bad_cell;     // min flat index of a non-physical cell
  // min flat index of a non-physical cell of the state a cycle ended with, found by the
  // update that also formed that state's primitives; it becomes the error when the next
  // cycle starts, where the primitive recovery of the split kernels would have found it
  unsigned long long bad_next;
  long long nsteps;
  int done;
  int err;
  int clamped;
  int pad;
};

struct Geo {
  int n[3];        // nx, ny, nz
  int stride[3];   // 1, nx, nx*ny
  int ncell;
  int active[3];   // n_d > 1
  double inv_dl[3];
  double dl[3];      // cell sizes l / n (the strict-rounding build divides by them)
  double gamma;
  double gm1;        // gamma - 1
  double gm1inv;     // 1 / (gamma - 1)
  float inv_dlf[3];  // 1/dl in FP32 for the FP32-bulk arithmetic
  float gammaf, gm1invf;
  int riemann;       // 1 Rusanov, 2 HLL, 4 HLLD
  int recon;         // 1 PLM (van Leer), 3 LimO3
  // floor(c / nx) and floor(c / (nx ny)) for 0 <= c < 2^31 as (c m) >> s (divmagic.cuh)
  unsigned div_m[2];
  int div_s[2];
};

inline void geo_set_divisors(Geo& g) {
  div_magic((unsigned)g.n[0], g.div_m[0], g.div_s[0]);
  div_magic((unsigned)g.stride[2], g.div_m[1], g.div_s[1]);
}

// gamma and 1/(gamma - 1) in the bulk type, formed once on the host
template <typename T> __device__ __forceinline__ T geo_gamma(const Geo& g);
template <> __device__ __forceinline__ double geo_gamma<double>(const Geo& g) { return g.gamma; }
template <> __device__ __forceinline__ float geo_gamma<float>(const Geo& g) { return g.gammaf; }
template <typename T> __device__ __forceinline__ T geo_gm1inv(const Geo& g);
template <> __device__ __forceinline__ double geo_gm1inv<double>(const Geo& g) { return g.gm1inv; }
template <> __device__ __forceinline__ float geo_gm1inv<float>(const Geo& g) { return g.gm1invf; }

// The derived constants of Geo.
inline void geo_set_gamma(Geo& geo, double gamma) {
  geo.gamma = gamma;
  geo.gm1 = gamma - 1.0;
  geo.gm1inv = 1.0 / (gamma - 1.0);
  geo.gammaf = (float)gamma;
  geo.gm1invf = (float)geo.gm1inv;
}

template <typename T> struct Ptr8 {
  T* f[8];
};

// Cell-centre EMF components -(v x B)_e of every cell, formed once per stage by the
// primitive recovery for the E^c kernel (each cell's value serves the 4 edges around it
// in each of 3 directions).  Null pointers: the E^c kernel forms them itself.
template <typename T> struct CellEmf {
  T* f[3];
};

// FP64 value into the bulk type and back, through the integer-pipe conversions for FP32.
template <typename T> __device__ __forceinline__ T to_bulk(double x);
template <> __device__ __forceinline__ double to_bulk<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_bulk<float>(double x) { return d2f_warp(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d(x); }

__device__ __forceinline__ void coords(const Geo& g, int c, int& i, int& j, int& k) {
  k = (int)div_by_magic((uint32_t)c, g.div_m[1], g.div_s[1]);
  const int r = c - k * g.stride[2];
  j = (int)div_by_magic((uint32_t)r, g.div_m[0], g.div_s[0]);
  i = r - j * g.n[0];
}

// Cell index shifted by s (|s| <= 2) along d with periodic wrap; needs n_d >= 2 for
// |s| == 2 and n_d >= 1 for |s| <= 1.
__device__ __forceinline__ int shifted(const Geo& g, int c, int coord, int d, int s) {
  int q = coord + s;
  const int n = g.n[d];
  if (q < 0) q += n;
  if (q < 0) q += n;
  if (q >= n) q -= n;
  if (q >= n) q -= n;
  return c + (q - coord) * g.stride[d];
}

// Offsets from a cell at coordinates ijk to its upper neighbour along each direction
// (periodic wrap; 0 along a one-cell direction).
__device__ __forceinline__ void upper_offsets(const Geo& g, const int ijk[3], int up[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) up[d] = (ijk[d] + 1 < g.n[d] ? 1 : 1 - g.n[d]) * g.stride[d];
}
// Offsets from cell c to its lower neighbour along each direction (periodic wrap).
__device__ __forceinline__ void lower_offsets(const Geo& g, int c, int dn[3]) {
  int ijk[3];
  coords(g, c, ijk[0], ijk[1], ijk[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) dn[d] = (ijk[d] > 0 ? 0 : g.n[d]) - 1;
#pragma unroll
  for (int d = 0; d < 3; ++d) dn[d] *= g.stride[d];
}

__device__ __forceinline__ void flag_bad(Ctrl* ctrl, int c) {
  atomicCAS(&ctrl->err, 0, IDX_ENONPHYS);
  atomicMin(&ctrl->bad_cell, (unsigned long long)c);
}
__device__ __forceinline__ void flag_bad_next(Ctrl* ctrl, int c) {
  atomicMin(&ctrl->bad_next, (unsigned long long)c);
}

// FP32-bulk primitive recovery of cell c from its FP64 conserved values (rho, m, E)
// and its six face fields (lower and upper face per direction), held in registers;
// writes W and the cell-centre EMFs and returns true for a non-physical cell.
__device__ __forceinline__ bool prims_f32_vals(const Geo& g, double rho, double mx, double my,
                                               double mz, double en, double bx0,
                                               double bx1, double by0, double by1,
                                               double bz0, double bz1,
                                               const Ptr8<float>& W,
                                               const CellEmf<float>& cc, int c) {
  // The velocities and cell-centre B go out in FP32; the pressure keeps FP64 accuracy.  Where every lane's rho, m and face B lie in [2^-32, 2^32) (or are
  // 0), the kinetic and magnetic energies are formed in double-float arithmetic on the
  // FP32 pipe (each input split exactly into 24 + 23 bits; error-free products and
  // sums; ~2^-46 relative) and only the cancellation E - K - M and the factor
  // (gamma - 1) take FP64 operations, 3 per cell.  Elsewhere all of it is FP64.
  const bool in_range = df_in_range(rho) & df_in_range(mx) & df_in_range(my) &
                        df_in_range(mz) & df_in_range(bx0) & df_in_range(bx1) &
                        df_in_range(by0) & df_in_range(by1) & df_in_range(bz0) &
                        df_in_range(bz1);
  double P;
  float rhof, irf, vx, vy, vz, bx, by, bz;
  if (__all_sync(__activemask(), in_range)) {
    const DF rd = df_split(rho), mxd = df_split(mx), myd = df_split(my), mzd = df_split(mz);
    // 1/rho: the FP32 reciprocal y of the high part, one Newton-Raphson step on the
    // double-float rho: 1/rho = y (1 + r) + O(r^2), r = 1 - rho y
    const float y = __frcp_rn(rd.h);
    const float r = __fmaf_rn(-rd.l, y, __fmaf_rn(-rd.h, y, 1.0f));
    const float yr = __fmul_rn(y, r);
    const DF ir2 = {0.5f * y, 0.5f * yr};  // 1 / (2 rho)
    const DF sx = df_add(df_split(bx0), df_split(bx1));  // 2 B_c
    const DF sy = df_add(df_split(by0), df_split(by1));
    const DF sz = df_add(df_split(bz0), df_split(bz1));
    const DF kin = df_mul(df_sum3(df_sqr(mxd), df_sqr(myd), df_sqr(mzd)), ir2);
    const DF ssq = df_sum3(df_sqr(sx), df_sqr(sy), df_sqr(sz));
    const DF km = df_add(kin, DF{0.125f * ssq.h, 0.125f * ssq.l});  // K + |B_c|^2 / 2
    P = g.gm1 * ((en - f2d_warp(km.h)) - f2d_warp(km.l));
    rhof = __fadd_rn(rd.h, rd.l);
    irf = __fadd_rn(y, yr);
    vx = __fadd_rn(mxd.h, mxd.l) * irf;
    vy = __fadd_rn(myd.h, myd.l) * irf;
    vz = __fadd_rn(mzd.h, mzd.l) * irf;
    bx = 0.5f * __fadd_rn(sx.h, sx.l);
    by = 0.5f * __fadd_rn(sy.h, sy.l);
    bz = 0.5f * __fadd_rn(sz.h, sz.l);
  } else {
    // 1/rho only scales the kinetic energy: an FP32 seed refined by one Newton-Raphson
    // step y1 = y0 + y0 (1 - rho y0) in FP64 (taken on y0/2, giving 1/(2 rho))
    rhof = d2f_warp(rho);
    const float y0f = __frcp_rn(rhof);
    const double y0h = f2d(0.5f * y0f);
    const double irh = fma(y0h, fma(-rho, f2d(y0f), 1.0), y0h);
    const double sx = bx0 + bx1, sy = by0 + by1, sz = bz0 + bz1;  // 2 B_c
    // P = (gamma - 1) (E - |m|^2 / (2 rho) - |2 B_c|^2 / 8), FP64 with fused steps
    const double msq = fma(mx, mx, fma(my, my, mz * mz));
    const double ssq = fma(sx, sx, fma(sy, sy, sz * sz));
    P = g.gm1 * fma(-0.125, ssq, fma(-msq, irh, en));
    irf = 2.0f * d2f_warp(irh);
    vx = d2f_warp(mx) * irf; vy = d2f_warp(my) * irf; vz = d2f_warp(mz) * irf;
    bx = 0.5f * d2f_warp(sx); by = 0.5f * d2f_warp(sy); bz = 0.5f * d2f_warp(sz);
  }
  // 0 < rho, P < infinity, tested on the bit patterns (FP64 compares take FP64 slots)
  const bool bad =
      !pos_finite(rho) || !pos_finite(P) || !isfinite(vx) || !isfinite(vy) || !isfinite(vz);
  W.f[0][c] = rhof; W.f[1][c] = vx; W.f[2][c] = vy; W.f[3][c] = vz;
  W.f[4][c] = d2f_warp(P);
  W.f[5][c] = bx; W.f[6][c] = by; W.f[7][c] = bz;
  if (cc.f[0]) {
    cc.f[0][c] = -(vy * bz - vz * by);
    cc.f[1][c] = -(vz * bx - vx * bz);
    cc.f[2][c] = -(vx * by - vy * bx);
  }
  return bad;
}

// ---------------------------------------------------------------------------
// Primitive recovery: rho, v = m/rho, P from E (at FP64 accuracy in both variants), and
// the cell-centre B as the mean of the two bounding faces.  W is stored as T.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void prims_body(const Geo& g, const Ptr8<const double>& U,
                                           const Ptr8<T>& W, const CellEmf<T>& cc, Ctrl* ctrl,
                                           int c) {
  int i, j, k;
  coords(g, c, i, j, k);
  const double rho = U.f[0][c];
  if constexpr (std::is_same<T, double>::value) {
    const double ir = 1.0 / rho;
    const double vx = U.f[1][c] * ir, vy = U.f[2][c] * ir, vz = U.f[3][c] * ir;
    const double bx = 0.5 * (U.f[5][c] + U.f[5][shifted(g, c, i, 0, 1)]);
    const double by = 0.5 * (U.f[6][c] + U.f[6][shifted(g, c, j, 1, 1)]);
    const double bz = 0.5 * (U.f[7][c] + U.f[7][shifted(g, c, k, 2, 1)]);
    const double kin = 0.5 * rho * (vx * vx + vy * vy + vz * vz);
    const double mag = 0.5 * (bx * bx + by * by + bz * bz);
    const double P = g.gm1 * (U.f[4][c] - kin - mag);
    // 0 < rho, P < infinity and finite velocities, on the bit patterns
    if (!pos_finite(rho) || !pos_finite(P) || !finite_bits(vx) || !finite_bits(vy) ||
        !finite_bits(vz))
      flag_bad(ctrl, c);
    W.f[0][c] = rho; W.f[1][c] = vx; W.f[2][c] = vy; W.f[3][c] = vz;
    W.f[4][c] = P;   W.f[5][c] = bx; W.f[6][c] = by; W.f[7][c] = bz;
    if (cc.f[0]) {
      cc.f[0][c] = -(vy * bz - vz * by);
      cc.f[1][c] = -(vz * bx - vx * bz);
      cc.f[2][c] = -(vx * by - vy * bx);
    }
  } else {
    const double mx = U.f[1][c], my = U.f[2][c], mz = U.f[3][c];
    const double bx0 = U.f[5][c], bx1 = U.f[5][shifted(g, c, i, 0, 1)];
    const double by0 = U.f[6][c], by1 = U.f[6][shifted(g, c, j, 1, 1)];
    const double bz0 = U.f[7][c], bz1 = U.f[7][shifted(g, c, k, 2, 1)];
    if (prims_f32_vals(g, rho, mx, my, mz, U.f[4][c], bx0, bx1, by0, by1, bz0, bz1, W, cc, c))
      flag_bad(ctrl, c);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 6 : 8) k_prims(Geo g, Ptr8<const double> U, Ptr8<T> W,
                                                    CellEmf<T> cc, Ctrl* ctrl, int check_dt) {
  if (check_dt && !(ctrl->dt > 0.0)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.ncell) prims_body<T>(g, U, W, cc, ctrl, c);
}

// Conserved state from primitives (cell-centre rho, v, P; face B).
__global__ void __launch_bounds__(kThreads) k_cons_from_prims(Geo g, Ptr8<const double> P,
                                                              Ptr8<double> U) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int i, j, k;
  coords(g, c, i, j, k);
  const double rho = P.f[0][c], vx = P.f[1][c], vy = P.f[2][c], vz = P.f[3][c];
  const double bx = 0.5 * (P.f[5][c] + P.f[5][shifted(g, c, i, 0, 1)]);
  const double by = 0.5 * (P.f[6][c] + P.f[6][shifted(g, c, j, 1, 1)]);
  const double bz = 0.5 * (P.f[7][c] + P.f[7][shifted(g, c, k, 2, 1)]);
  U.f[0][c] = rho;
  U.f[1][c] = rho * vx;
  U.f[2][c] = rho * vy;
  U.f[3][c] = rho * vz;
  U.f[4][c] = P.f[4][c] / g.gm1 + 0.5 * rho * (vx * vx + vy * vy + vz * vz) +
              0.5 * (bx * bx + by * by + bz * bz);
  U.f[5][c] = P.f[5][c];
  U.f[6][c] = P.f[6][c];
  U.f[7][c] = P.f[7][c];
}

// ---------------------------------------------------------------------------
// Non-periodic boundaries.  Along a non-periodic direction the grid carries two ghost
// cells per side (interior cell i is cell i + 2; the normal field's n + 1 faces are faces
// 2 .. n + 2) and is stepped as a periodic one: the wrap-around only touches ghost cells,
// which k_fill_ghosts refills from the interior before every stage, direction by
// direction (x, y, z, each over the full padded extent of the others, so edge and corner
// ghosts are consistent).  Outflow: copies of the nearest interior cell (cell fields and
// the transverse face fields stored with it) and of the boundary face (normal field).
// Reflecting: the mirror image about the boundary face with the normal momentum and
// normal field reversed.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_fill_ghosts(Geo g, int d, int kind,
                                                          Ptr8<double> U) {
  const int a = (d + 1) % 3, b = (d + 2) % 3;
  const long long total = 4ll * g.n[a] * g.n[b];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int slot = (int)(t & 3);
  const long long r = t >> 2;
  const int oa = (int)(r % g.n[a]), ob = (int)(r / g.n[a]);
  const int n = g.n[d] - 4;  // interior cells
  const int base = oa * g.stride[a] + ob * g.stride[b];
  const int sd = g.stride[d];
  const int gp = slot < 2 ? slot : n + slot;  // ghost cells 0, 1, n + 2, n + 3
  const bool reflect = kind == IDX_BC_REFLECTING;
  const int src = reflect ? (slot < 2 ? 3 - gp : 2 * n + 3 - gp) : (slot < 2 ? 2 : n + 1);
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    if (f == 5 + d) continue;
    const double v = U.f[f][base + src * sd];
    U.f[f][base + gp * sd] = (reflect && f == 1 + d) ? -v : v;
  }
  // normal field on the ghost faces 0, 1 and n + 3 (face n + 2 is the boundary face)
  if (slot == 2) return;
  const int fsrc = reflect ? (slot == 0 ? 4 : (slot == 1 ? 3 : n + 1)) : (slot < 2 ? 2 : n + 2);
  const double v = U.f[5 + d][base + fsrc * sd];
  U.f[5 + d][base + gp * sd] = reflect ? -v : v;
}

// User layout <-> padded layout of the 8 fields (user layout: cells n_d, the normal field
// n_d + 1 faces along a non-periodic d).  One thread per point of the user box extended
// by one along each non-periodic direction.
struct Pad {
  int un[3];    // user cells per direction
  int off[3];   // 2 along a non-periodic direction, else 0
  int ext[3];   // 1 along a non-periodic direction, else 0
};
__global__ void __launch_bounds__(kThreads) k_pad(Geo g, Pad pd, Ptr8<const double> src,
                                                  Ptr8<double> dst, int unpad) {
  const int ex = pd.un[0] + pd.ext[0], ey = pd.un[1] + pd.ext[1], ez = pd.un[2] + pd.ext[2];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ex * ey * ez) return;
  const int i = (int)(t % ex);
  const long long r = t / ex;
  const int j = (int)(r % ey), k = (int)(r / ey);
  const int p = (i + pd.off[0]) + (j + pd.off[1]) * g.stride[1] + (k + pd.off[2]) * g.stride[2];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    // this field's user extent: the normal field of a non-periodic direction has n + 1
    const int ux = pd.un[0] + (f == 5 ? pd.ext[0] : 0);
    const int uy = pd.un[1] + (f == 6 ? pd.ext[1] : 0);
    const int uz = pd.un[2] + (f == 7 ? pd.ext[2] : 0);
    if (i >= ux || j >= uy || k >= uz) continue;
    const long long u = i + (long long)ux * (j + (long long)uy * k);
    if (unpad) dst.f[f][u] = src.f[f][p];
    else dst.f[f][p] = src.f[f][u];
  }
}

// ---------------------------------------------------------------------------
// Sweep along direction D: a thread owns a segment of up to SEG faces of one pencil,
// marches along D keeping three cells' primitives and one slope in registers, and
// computes each cell's van Leer slopes once and each face's HLLD flux once.
// Face f of a pencil is the lower D-face of cell f.  Output (rotated order): F[0..6]
// = fluxes of rho, m_n, m_t1, m_t2, E, B_t1, B_t2 with t1 = D+1, t2 = D+2; F[7] = c.
// ---------------------------------------------------------------------------
// number of threads of a marching sweep of direction d with segment seg
__host__ __device__ __forceinline__ int march_threads(const Geo& g, int d, int seg) {
  return g.n[(d + 1) % 3] * g.n[(d + 2) % 3] * ((g.n[d] + seg - 1) / seg);
}

// SPEEDS: the signal-speed pass -- reconstruct and form only the face's c (slot 7).
// RECON: 1 PLM with the van Leer limiter, 3 LimO3 (Sec. 2.3); both read cells f-2 .. f+1.
template <typename T, int D, int SEG, bool SPEEDS = false, int RECON = 1>
__device__ __forceinline__ void sweep_body(const Geo& g, const Ptr8<const T>& W,
                                           const double* bface, const Ptr8<T>& F, int t) {
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  const int nd = g.n[D];
  const int npencil = g.n[A] * g.n[B];
  const int nseg = (nd + SEG - 1) / SEG;
  if (t >= npencil * nseg) return;
  const int pencil = t % npencil, seg = t / npencil;
  // pencil -> coordinates of the two other directions, x fastest for coalescing
  int cA, cB;
  if (D == 0) {  // other dims y (A), z (B)
    cA = pencil % g.n[1]; cB = pencil / g.n[1];
  } else if (D == 1) {  // A = z, B = x: x fastest
    cB = pencil % g.n[0]; cA = pencil / g.n[0];
  } else {  // D == 2: A = x, B = y
    cA = pencil % g.n[0]; cB = pencil / g.n[0];
  }
  const int base = cA * g.stride[A] + cB * g.stride[B];
  const int sd = g.stride[D];
  const int f0 = seg * SEG;
  const int f1 = min(f0 + SEG, nd);
  auto cell = [&](int q) {  // flat index of cell q (wrapped) along the pencil
    q = (q < 0) ? q + nd : q;
    q = (q < 0) ? q + nd : q;
    q = (q >= nd) ? q - nd : q;
    q = (q >= nd) ? q - nd : q;
    return base + q * sd;
  };
  // rotated variable slots in W: rho, v_n, v_t1, v_t2, P, B_t1, B_t2; the speed-only pass
  // reconstructs the 5 that the outer speeds use (rho, v_n, P, B_t1, B_t2)
  constexpr int NV = SPEEDS ? 5 : 7;
  constexpr int var[7] = {0, 1 + D, SPEEDS ? 4 : 1 + A, SPEEDS ? 5 + A : 1 + B,
                          SPEEDS ? 5 + B : 4, 5 + A, 5 + B};
  const T gamma = geo_gamma<T>(g);
  const T gm1inv = geo_gm1inv<T>(g);

  // cells f-1, f, f+1 in registers, cell f+2 prefetched one face ahead so that its
  // loads overlap the current face's Riemann solve.  slope_m: the change of cell f-1 at
  // its upper face (face f); slope0: the change of cell f at its lower face, subtracted.
  // PLM uses one half slope for both faces of a cell; LimO3 has one per face.
  T wm[7], w0[7], wp[7], wn[7], slope_m[7];
  {
    const int cm2 = cell(f0 - 2), cm1 = cell(f0 - 1), c0 = cell(f0), cp = cell(f0 + 1);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const T a = W.f[var[q]][cm2];
      wm[q] = W.f[var[q]][cm1];
      w0[q] = W.f[var[q]][c0];
      wp[q] = W.f[var[q]][cp];
      slope_m[q] = RECON == 3 ? limo3_half(wm[q] - a, w0[q] - wm[q])
                              : vanleer_half(wm[q] - a, w0[q] - wm[q]);
    }
  }
  for (int f = f0; f < f1; ++f) {
    const int cf = cell(f);
    if (f + 1 < f1) {
      const int cn = cell(f + 2);
#pragma unroll
      for (int q = 0; q < NV; ++q) wn[q] = W.f[var[q]][cn];
    }
    Side<T> L, R;
    T slope0[7], up0[7];
    if constexpr (RECON == 3) {
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const T dl = w0[q] - wm[q], dr = wp[q] - w0[q];
        slope0[q] = limo3_half(dr, dl);
        up0[q] = limo3_half(dl, dr);
      }
    } else {
      T dl[NV], dr[NV];
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        dl[q] = w0[q] - wm[q];
        dr[q] = wp[q] - w0[q];
      }
      vanleer_half_n<NV>(dl, dr, slope0);
#pragma unroll
      for (int q = 0; q < NV; ++q) up0[q] = slope0[q];
    }
    if constexpr (SPEEDS) {
      L.r = wm[0] + slope_m[0]; R.r = w0[0] - slope0[0];
      L.u = wm[1] + slope_m[1]; R.u = w0[1] - slope0[1];
      L.v = L.w = R.v = R.w = T(0);  // the outer speeds do not use the transverse velocity
      L.p = wm[2] + slope_m[2]; R.p = w0[2] - slope0[2];
      L.b1 = wm[3] + slope_m[3]; R.b1 = w0[3] - slope0[3];
      L.b2 = wm[4] + slope_m[4]; R.b2 = w0[4] - slope0[4];
    } else {
      L.r = wm[0] + slope_m[0]; R.r = w0[0] - slope0[0];
      L.u = wm[1] + slope_m[1]; R.u = w0[1] - slope0[1];
      L.v = wm[2] + slope_m[2]; R.v = w0[2] - slope0[2];
      L.w = wm[3] + slope_m[3]; R.w = w0[3] - slope0[3];
      L.p = wm[4] + slope_m[4]; R.p = w0[4] - slope0[4];
      L.b1 = wm[5] + slope_m[5]; R.b1 = w0[5] - slope0[5];
      L.b2 = wm[6] + slope_m[6]; R.b2 = w0[6] - slope0[6];
    }
    const T bn = to_bulk<T>(bface[cf]);
    if constexpr (SPEEDS) {
      F.f[7][cf] = outer_speed(g.riemann, L, R, bn, gamma);
    } else {
      T flux[7], cmax;
      riemann_flux(g.riemann, L, R, bn, gamma, gm1inv, flux, cmax);
#pragma unroll
      for (int q = 0; q < 7; ++q) F.f[q][cf] = flux[q];
      F.f[7][cf] = cmax;
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      wm[q] = w0[q];
      w0[q] = wp[q];
      wp[q] = wn[q];
      slope_m[q] = up0[q];
    }
  }
}

template <typename T, int D, int SEG, int RECON = 1>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 1)
    k_sweep(Geo g, Ptr8<const T> W, const double* bface,
                                                    Ptr8<T> F, const Ctrl* ctrl, int check_dt) {
  if (check_dt && !(ctrl->dt > 0.0)) return;
  sweep_body<T, D, SEG, false, RECON>(g, W, bface, F, blockIdx.x * blockDim.x + threadIdx.x);
}

// Signal speeds of one direction for the first dt of a new state (16-face segments).
template <typename T, int D, int RECON>
__global__ void __launch_bounds__(kThreads) k_sweep_speeds(Geo g, Ptr8<const T> W,
                                                           const double* bface, Ptr8<T> F) {
  sweep_body<T, D, 16, true, RECON>(g, W, bface, F, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// TMA-staged sweep along D = y or z.  A block owns a tile of 32 x-cells by L faces
// along D at one coordinate of the third direction.  One thread copies the tile's
// primitives (the 7 rotated variables, L cells plus a 2-cell periodic halo on each
// side) from HBM into shared memory with bulk tensor copies -- body, low halo and high
// halo as separate boxes, so every coordinate is in range and wraps by hand -- and the
// block waits on an mbarrier (bounded).  Then warp w marches faces 4w..4w+3 of the tile
// from shared memory, lane = x, with the same per-face arithmetic as k_sweep.  The
// global loads of a marching thread wait ~1 us each; here a tile's loads are in flight
// together and the march reads shared memory.
// Tile shapes: L = 16 (128 threads) or 32 (256 threads); nx % 32 == 0, n_D % L == 0.
// ---------------------------------------------------------------------------
constexpr uint64_t kWaitNs = 50000000ull;  // bounded mbarrier wait: 50 ms, ~10^4 x a tile copy

__device__ __forceinline__ void flag_timeout(Ctrl* ctrl) {
  atomicCAS(&ctrl->err, 0, IDX_ETIMEOUT);
}

// One staged tile: tile index -> (x tile, D tile, coordinate along the third direction),
// copies issued by thread 0 onto `bar`, bounded wait for the phase of parity `parity`,
// then the march.  Returns false (the same on every thread of the block) if the copies
// did not land in time; the caller then records the timeout and leaves.  RECON as in
// sweep_body (1 PLM, 3 LimO3).
template <typename T, int D, int L, int RECON = 1>
__device__ __forceinline__ bool tma_tile(const Geo& g, const CUtensorMap* tm_body,
                                         const CUtensorMap* tm_halo, const double* bface,
                                         const Ptr8<T>& F, int tile_index, T* tile,
                                         uint64_t* bar, uint32_t parity) {
  static_assert(D == 1 || D == 2, "staged sweeps run along y or z");
  constexpr int A = (D + 1) % 3, B = (D + 2) % 3;
  constexpr int ROWS = L + 4, PLANE = ROWS * 32;
  constexpr int O = (D == 1) ? 2 : 1;  // the transverse direction that is not x
  const int ntx = g.n[0] >> 5, ntd = g.n[D] / L;
  int b = tile_index;
  const int x0 = (b % ntx) * 32;
  b /= ntx;
  const int t0 = (b % ntd) * L;
  const int co = b / ntd;  // coordinate along O
  // rotated variable slots of W: rho, v_n, v_t1, v_t2, P, B_t1, B_t2
  constexpr int var[7] = {0, 1 + D, 1 + A, 1 + B, 4, 5 + A, 5 + B};

  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, 7u * PLANE * sizeof(T));
    int lo = t0 - 2;
    if (lo < 0) lo += g.n[D];
    int hi = t0 + L;
    if (hi >= g.n[D]) hi -= g.n[D];
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      T* dst = tile + q * PLANE;
      if (D == 1) {
        tma_load_4d(dst, tm_halo, x0, lo, co, var[q], bar);
        tma_load_4d(dst + 2 * 32, tm_body, x0, t0, co, var[q], bar);
        tma_load_4d(dst + (L + 2) * 32, tm_halo, x0, hi, co, var[q], bar);
      } else {
        tma_load_4d(dst, tm_halo, x0, co, lo, var[q], bar);
        tma_load_4d(dst + 2 * 32, tm_body, x0, co, t0, var[q], bar);
        tma_load_4d(dst + (L + 2) * 32, tm_halo, x0, co, hi, var[q], bar);
      }
    }
  }
  const int lane = threadIdx.x & 31, f0 = (threadIdx.x >> 5) * 4;
  // flat index of the cell whose lower D-face is face f of the tile
  const int cbase = x0 + lane + co * g.stride[O];
  T bn[4];  // the Riemann solves take the normal field in the bulk type
#pragma unroll
  for (int q = 0; q < 4; ++q) bn[q] = to_bulk<T>(bface[cbase + (t0 + f0 + q) * g.stride[D]]);
  const bool landed = mbar_wait(bar, parity, kWaitNs);
  if (__syncthreads_or(!landed)) return false;
  const T gamma = geo_gamma<T>(g);
  const T gm1inv = geo_gm1inv<T>(g);
  auto ld = [&](int q, int row) { return tile[q * PLANE + row * 32 + lane]; };
  // face f uses tile rows f .. f+3 (cells f-2 .. f+1); slope_m: the change of cell f-1 at
  // face f, slope0: the change of cell f at face f (subtracted), up0: at face f+1
  T wm[7], w0[7], wp[7], slope_m[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const T a = ld(q, f0);
    wm[q] = ld(q, f0 + 1);
    w0[q] = ld(q, f0 + 2);
    wp[q] = ld(q, f0 + 3);
    slope_m[q] = RECON == 3 ? limo3_half(wm[q] - a, w0[q] - wm[q])
                            : vanleer_half(wm[q] - a, w0[q] - wm[q]);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Side<T> Ls, Rs;
    T slope0[7], up0[7];
    if constexpr (RECON == 3) {
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        const T dl = w0[q] - wm[q], dr = wp[q] - w0[q];
        slope0[q] = limo3_half(dr, dl);
        up0[q] = limo3_half(dl, dr);
      }
    } else {
      T dl[7], dr[7];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        dl[q] = w0[q] - wm[q];
        dr[q] = wp[q] - w0[q];
      }
      vanleer_half7(dl, dr, slope0);
#pragma unroll
      for (int q = 0; q < 7; ++q) up0[q] = slope0[q];
    }
    Ls.r = wm[0] + slope_m[0]; Rs.r = w0[0] - slope0[0];
    Ls.u = wm[1] + slope_m[1]; Rs.u = w0[1] - slope0[1];
    Ls.v = wm[2] + slope_m[2]; Rs.v = w0[2] - slope0[2];
    Ls.w = wm[3] + slope_m[3]; Rs.w = w0[3] - slope0[3];
    Ls.p = wm[4] + slope_m[4]; Rs.p = w0[4] - slope0[4];
    Ls.b1 = wm[5] + slope_m[5]; Rs.b1 = w0[5] - slope0[5];
    Ls.b2 = wm[6] + slope_m[6]; Rs.b2 = w0[6] - slope0[6];
    T flux[7], cmax;
    riemann_flux(g.riemann, Ls, Rs, bn[k], gamma, gm1inv, flux, cmax);
    const int cf = cbase + (t0 + f0 + k) * g.stride[D];
#pragma unroll
    for (int q = 0; q < 7; ++q) F.f[q][cf] = flux[q];
    F.f[7][cf] = cmax;
    if (k < 3) {
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        wm[q] = w0[q];
        w0[q] = wp[q];
        wp[q] = ld(q, f0 + k + 4);
        slope_m[q] = up0[q];
      }
    }
  }
  return true;
}

// After a timeout: record it, give the copies in flight a bounded time to land in
// shared memory, and let the block leave.
__device__ __forceinline__ void tma_give_up(Ctrl* ctrl, uint64_t* bar, uint32_t parity) {
  if (threadIdx.x == 0) flag_timeout(ctrl);
  mbar_wait(bar, parity, kWaitNs);
}

template <typename T, int D, int L, int RECON = 1>
__global__ void __launch_bounds__(8 * L, sizeof(T) == 4 ? 96 / L : 1)
    k_sweep_tma(Geo g, const __grid_constant__ CUtensorMap tm_body,
                const __grid_constant__ CUtensorMap tm_halo, const double* bface, Ptr8<T> F,
                Ctrl* ctrl, int check_dt) {
  if (check_dt && !(ctrl->dt > 0.0)) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);  // [7][L + 4][32]: variable, row along D, x
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (!tma_tile<T, D, L, RECON>(g, &tm_body, &tm_halo, bface, F, blockIdx.x, tile, &bar, 0))
    tma_give_up(ctrl, &bar, 0);
}

// ---------------------------------------------------------------------------
// TMA-staged sweep along x.  A block owns 32 x-faces of 8 consecutive y-rows at one z.
// Each of the 7 rotated variables arrives as one bulk tensor copy of 40 x 8 cells, the
// 32 cells of the rows with 4 more on each side (the start of a copy must sit on a
// 16-byte boundary, so the 2-cell halo is fetched 4 wide).  Where the box runs past an
// end of the row the copy fills zeros and the block patches those 4 columns with the
// periodic images by plain loads.  Warp r takes row r, lane f face f: it forms the slope
// of cell f once, keeps w - slope as the face's right state and hands w + slope to lane
// f + 1 as that face's left state; the left state of face 0 (cell -1, one per row) is
// formed beforehand by 56 threads, one per (row, variable).  Needs nx % 32 == 0 and
// ny % 8 == 0.
// ---------------------------------------------------------------------------
constexpr int kXRows = 8;
constexpr int kXBox = 40;   // cells per row in the staged box: 4 + 32 + 4

template <typename T>
__global__ void __launch_bounds__(32 * kXRows)
    k_sweep_tma_x(Geo g, const __grid_constant__ CUtensorMap tm_row, Ptr8<const T> W,
                  const double* bface, Ptr8<T> F, Ctrl* ctrl, int check_dt) {
  if (check_dt && !(ctrl->dt > 0.0)) return;
  constexpr int R = kXRows;
  constexpr int PLANE = R * kXBox;
  __shared__ __align__(128) T tile[7 * PLANE];     // [var][row][col], col = x - x0 + 4
  __shared__ T left0[7][R];                         // left state of face 0 per row
  __shared__ __align__(8) uint64_t bar;
  const int nx = g.n[0];
  const int ntx = nx >> 5, nty = g.n[1] / R;
  int b = blockIdx.x;
  const int x0 = (b % ntx) * 32;
  b /= ntx;
  const int y0 = (b % nty) * R;
  const int z = b / nty;
  constexpr int var[7] = {0, 1, 2, 3, 4, 6, 7};  // rho, v_n = vx, vy, vz, P, B_t1 = By, B_t2 = Bz
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(&bar, 7u * PLANE * sizeof(T));
#pragma unroll
    for (int q = 0; q < 7; ++q) tma_load_4d(tile + q * PLANE, &tm_row, x0 - 4, y0, z, var[q], &bar);
  }
  const int f = threadIdx.x & 31, r = threadIdx.x >> 5;
  const int c = (x0 + f) + (y0 + r) * g.stride[1] + z * g.stride[2];
  const T bn = to_bulk<T>(bface[c]);
  const bool landed = mbar_wait(&bar, 0, kWaitNs);
  if (__syncthreads_or(!landed)) {
    tma_give_up(ctrl, &bar, 0);
    return;
  }
  // periodic images of the columns the copy filled with zeros (block-uniform branches)
  const bool wrap_lo = x0 == 0, wrap_hi = x0 + 32 == nx;
  if (wrap_lo || wrap_hi) {
    // 8 rows x 4 columns per side, one thread each, all 7 variables
    if (threadIdx.x < 4 * R) {
      const int k = threadIdx.x & 3, row = threadIdx.x >> 2;
      const int rowoff = (y0 + row) * g.stride[1] + z * g.stride[2];
#pragma unroll
      for (int q = 0; q < 7; ++q) {
        T* dst = tile + q * PLANE + row * kXBox;
        if (wrap_lo) dst[k] = W.f[var[q]][rowoff + nx - 4 + k];
        if (wrap_hi) dst[36 + k] = W.f[var[q]][rowoff + k];
      }
    }
    __syncthreads();
  }
  // cell at column col (-4 .. 35) of row rr of variable q
  auto ld = [&](int q, int rr, int col) { return tile[q * PLANE + rr * kXBox + col + 4]; };
  if (threadIdx.x < 7 * R) {
    const int q = threadIdx.x / R, rr = threadIdx.x % R;
    const T wmm = ld(q, rr, -2), wm = ld(q, rr, -1), w0 = ld(q, rr, 0);
    left0[q][rr] = wm + vanleer_half(wm - wmm, w0 - wm);
  }
  __syncthreads();
  Side<T> Ls, Rs;
  T Lq[7], Rq[7], wc[7], dl[7], dr[7], hs[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const T wm = ld(q, r, f - 1), wp = ld(q, r, f + 1);
    wc[q] = ld(q, r, f);
    dl[q] = wc[q] - wm;
    dr[q] = wp - wc[q];
  }
  vanleer_half7(dl, dr, hs);   // FP64: the cell's 7 slopes share one reciprocal
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    Rq[q] = wc[q] - hs[q];
    const T up = __shfl_up_sync(0xffffffffu, wc[q] + hs[q], 1);
    Lq[q] = f == 0 ? left0[q][r] : up;
  }
  Ls.r = Lq[0]; Ls.u = Lq[1]; Ls.v = Lq[2]; Ls.w = Lq[3]; Ls.p = Lq[4]; Ls.b1 = Lq[5]; Ls.b2 = Lq[6];
  Rs.r = Rq[0]; Rs.u = Rq[1]; Rs.v = Rq[2]; Rs.w = Rq[3]; Rs.p = Rq[4]; Rs.b1 = Rq[5]; Rs.b2 = Rq[6];
  T flux[7], cmax;
  riemann_flux(g.riemann, Ls, Rs, bn, geo_gamma<T>(g), geo_gm1inv<T>(g), flux, cmax);
#pragma unroll
  for (int q = 0; q < 7; ++q) F.f[q][c] = flux[q];
  F.f[7][c] = cmax;
}

// ---------------------------------------------------------------------------
// Sweep along x: one warp per run of 32 consecutive cells of an x-row, lane l holding
// cell base + l (mod nx), so every load is coalesced.  A lane gets its neighbours'
// primitives and slopes by warp shuffle; lane 0 also loads cells base-1, base-2 and
// forms the slope of base-1, lane 31 loads cell base+32.  Each cell's slope is computed
// once (plus one per warp) and each face's HLLD once.
// ---------------------------------------------------------------------------
// threads of the warp x sweep (a multiple of 32)
__host__ __device__ __forceinline__ int warpx_threads(const Geo& g) {
  return g.n[1] * g.n[2] * ((g.n[0] + 31) / 32) * 32;
}

template <typename T>
__device__ __forceinline__ void sweep_x_body(const Geo& g, const Ptr8<const T>& W,
                                             const double* bface, const Ptr8<T>& F, int t) {
  const int nx = g.n[0];
  const int wpr = (nx + 31) >> 5;  // warps per x-row
  const int nrows = g.n[1] * g.n[2];
  const int warp = t >> 5;
  if (warp >= nrows * wpr) return;  // whole warps leave together
  const int lane = t & 31;
  const int row = warp / wpr;
  const int base = (warp - row * wpr) * 32;
  const int rowoff = row * nx;
  auto at_x = [&](int q) {
    q %= nx;
    return rowoff + (q < 0 ? q + nx : q);
  };
  const int i = base + lane;
  const int c = at_x(i);
  constexpr int var[7] = {0, 1, 2, 3, 4, 6, 7};  // rho, v_n = vx, vy, vz, P, B_t1 = By, B_t2 = Bz
  const T gamma = geo_gamma<T>(g);
  const T gm1inv = geo_gm1inv<T>(g);
  T w0[7], wm1[7], wm2[7], wp32[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) w0[q] = W.f[var[q]][c];
  if (lane == 0) {
    const int cm1 = at_x(base - 1), cm2 = at_x(base - 2);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      wm1[q] = W.f[var[q]][cm1];
      wm2[q] = W.f[var[q]][cm2];
    }
  }
  if (lane == 31) {
    const int cp = at_x(base + 32);
#pragma unroll
    for (int q = 0; q < 7; ++q) wp32[q] = W.f[var[q]][cp];
  }
  Side<T> L, R;
  T Lq[7], Rq[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    T up = __shfl_up_sync(0xffffffffu, w0[q], 1);    // cell c-1
    T dn = __shfl_down_sync(0xffffffffu, w0[q], 1);  // cell c+1
    if (lane == 0) up = wm1[q];
    if (lane == 31) dn = wp32[q];
    const T slope0 = vanleer_half(w0[q] - up, dn - w0[q]);
    T slope_m = __shfl_up_sync(0xffffffffu, slope0, 1);  // slope of cell c-1
    if (lane == 0) slope_m = vanleer_half(wm1[q] - wm2[q], w0[q] - wm1[q]);
    Lq[q] = up + slope_m;
    Rq[q] = w0[q] - slope0;
  }
  if (i >= nx) return;
  L.r = Lq[0]; L.u = Lq[1]; L.v = Lq[2]; L.w = Lq[3]; L.p = Lq[4]; L.b1 = Lq[5]; L.b2 = Lq[6];
  R.r = Rq[0]; R.u = Rq[1]; R.v = Rq[2]; R.w = Rq[3]; R.p = Rq[4]; R.b1 = Rq[5]; R.b2 = Rq[6];
  T flux[7], cmax;
  riemann_flux(g.riemann, L, R, to_bulk<T>(bface[c]), gamma, gm1inv, flux, cmax);
#pragma unroll
  for (int q = 0; q < 7; ++q) F.f[q][c] = flux[q];
  F.f[7][c] = cmax;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_sweep_x(Geo g, Ptr8<const T> W, const double* bface,
                                                      Ptr8<T> F, const Ctrl* ctrl, int check_dt) {
  if (check_dt && !(ctrl->dt > 0.0)) return;
  sweep_x_body<T>(g, W, bface, F, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Edge EMFs: E_e at the edge along e bounded by the lower a- and b-faces of cell c,
// a = e+1, b = e+2.  a-face EMF = -F_a[B_b] (rotated slot 5 of direction a), b-face
// EMF = +F_b[B_a] (slot 6 of direction b), cell-centre EMF = -(v_a B_b - v_b B_a).
// dn: the offsets from c to its lower neighbour along each direction (lower_offsets).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T edge_emf(const Geo& g, int e, int c, const int dn[3],
                                      const Ptr8<const T>& W, const Ptr8<const T>* F,
                                      const T* cce) {
  const int a = (e + 1) % 3, b = (e + 2) % 3;
  const Ptr8<const T>& Fa = F[a];
  const Ptr8<const T>& Fb = F[b];
  const int cb = c + dn[b];          // c - e_b
  const int ca = c + dn[a];          // c - e_a
  const int cab = c + dn[a] + dn[b];  // c - e_a - e_b
  const T X0 = -Fa.f[5][c], X1 = -Fa.f[5][cb];
  const T Y0 = Fb.f[6][c], Y1 = Fb.f[6][ca];
  const T Fa0 = Fa.f[0][c], Fa1 = Fa.f[0][cb];
  const T Fb0 = Fb.f[0][c], Fb1 = Fb.f[0][ca];
  auto cc = [&](int q) {
    return cce ? cce[q] : -(W.f[1 + a][q] * W.f[5 + b][q] - W.f[1 + b][q] * W.f[5 + a][q]);
  };
  const T C00 = cc(c), C01 = cc(cb), C10 = cc(ca), C11 = cc(cab);
#ifdef IDX_STRICT_ROUNDING
  if constexpr (sizeof(T) == 8)
    return emf_ec_plain(X0, X1, Y0, Y1, C00, C01, C10, C11, Fa0, Fa1, Fb0, Fb1, g.dl[a], g.dl[b]);
#endif
  return emf_ec(X0, X1, Y0, Y1, C00, C01, C10, C11, Fa0, Fa1, Fb0, Fb1);
}

template <typename T>
__device__ __forceinline__ void emf_body(const Geo& g, const Ptr8<const T>& W,
                                         const Ptr8<const T>& Fx, const Ptr8<const T>& Fy,
                                         const Ptr8<const T>& Fz, const CellEmf<T>& cc, T* Ex,
                                         T* Ey, T* Ez, int c) {
  int dn[3];
  lower_offsets(g, c, dn);
  const Ptr8<const T> F[3] = {Fx, Fy, Fz};
  T* out[3] = {Ex, Ey, Ez};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    if (g.active[a] && g.active[b]) out[e][c] = edge_emf<T>(g, e, c, dn, W, F, cc.f[e]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 8 : 1) k_emf(Geo g, Ptr8<const T> W, Ptr8<const T> Fx,
                                                  Ptr8<const T> Fy, Ptr8<const T> Fz,
                                                  CellEmf<T> cc, T* Ex, T* Ey, T* Ez,
                                                  const Ctrl* ctrl) {
  if (!(ctrl->dt > 0.0)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < g.ncell) emf_body<T>(g, W, Fx, Fy, Fz, cc, Ex, Ey, Ez, c);
}

// Rotated flux slot of conserved field f (0..4) or face field 5+m for direction d.
__device__ __forceinline__ int slot(int f, int d) {
  if (f == 0) return 0;
  if (f == 4) return 4;
  if (f <= 3) {  // momentum component m = f-1
    const int m = f - 1;
    return m == d ? 1 : (m == (d + 1) % 3 ? 2 : 3);
  }
  const int m = f - 5;  // field component, tangential to d
  return m == (d + 1) % 3 ? 5 : 6;
}

// ---------------------------------------------------------------------------
// Vector-potential form of the induction equation (Sec. 2.4, Eqs. 7-8).  The edge
// potential A sits where the edge EMF sits.  Per stage the EMF kernel steps it,
// A_out = w (A_in - dt E) + w0 A_0, instead of storing E, and the update kernel sets
// every face field to Bref + curl A_out (Stokes on the face) instead of stepping it.
// With one transverse direction of an edge not integrated, the edge collapses onto a
// face of the other one and the EMF there is the face flux of the field normal to
// the thin direction: E_e = -F_a[B_b] on an a-face, +F_b[B_a] on a b-face.
// ---------------------------------------------------------------------------
struct Ptr3 {
  double* f[3];
};

struct PotStage {
  const double* in[3];    // A of the stage input
  const double* a0[3];    // A at the start of the cycle (the w0 term)
  double* out[3];         // A of the stage output
  const double* bref[3];  // the fixed face field
};

template <typename T, bool COMBINE>
__global__ void __launch_bounds__(kThreads) k_emf_pot(Geo g, Ptr8<const T> W, Ptr8<const T> Fx,
                                                      Ptr8<const T> Fy, Ptr8<const T> Fz,
                                                      CellEmf<T> cc, PotStage P, const Ctrl* ctrl,
                                                      double w, double w0) {
  const double dt = ctrl->dt;
  if (!(dt > 0.0)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int dn[3];
  lower_offsets(g, c, dn);
  const Ptr8<const T> F[3] = {Fx, Fy, Fz};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int a = (e + 1) % 3, b = (e + 2) % 3;
    double E = 0.0;  // neither transverse direction integrated: A_e enters no face field
    if (g.active[a] && g.active[b]) E = to_f64(edge_emf<T>(g, e, c, dn, W, F, cc.f[e]));
    else if (g.active[a]) E = -to_f64(F[a].f[slot(5 + b, a)][c]);
    else if (g.active[b]) E = to_f64(F[b].f[slot(5 + a, b)][c]);
    const double As = P.in[e][c] - dt * E;
    P.out[e][c] = COMBINE ? fma(w, As, w0 * P.a0[e][c]) : As;
  }
}

// Face field = bmean + curl A, for a state given by its potential.  Also fills the
// fixed field Bref with bmean when bref is set.
struct Vec3 {
  double v[3];
};
__global__ void __launch_bounds__(kThreads) k_b_from_pot(Geo g, Ptr3 A, Vec3 bmean, Ptr3 B,
                                                         Ptr3 bref, int fill_bref) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int ijk[3];
  coords(g, c, ijk[0], ijk[1], ijk[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    double b = bmean.v[d];
    if (g.active[t1])
      b += (A.f[t2][shifted(g, c, ijk[t1], t1, 1)] - A.f[t2][c]) * g.inv_dl[t1];
    if (g.active[t2])
      b -= (A.f[t1][shifted(g, c, ijk[t2], t2, 1)] - A.f[t1][c]) * g.inv_dl[t2];
    B.f[d][c] = b;
    if (fill_bref) bref.f[d][c] = bmean.v[d];
  }
}

// ---------------------------------------------------------------------------
// Update: U* = U - dt div F (cell fields), B* = B - dt curl E (face fields, Eq. 6),
// U_out = w U* + w0 U_0 (Eq. 9), and the stage's inverse CFL time (Eq. 10).
// Arithmetic in FP64 for both variants.
// ---------------------------------------------------------------------------
// block-wide max of non-negative values, reduced in their own type, into *bits (the bit
// pattern of the max as a double: non-negative doubles order like their bit patterns)
template <typename V>
__device__ __forceinline__ void block_max_to(unsigned long long* bits, V v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max_nn(v, __shfl_xor_sync(0xffffffffu, v, o));
  __shared__ V wmax[kThreads / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    V m = wmax[0];
    for (int w = 1; w < kThreads / 32; ++w) m = max_nn(m, wmax[w]);
    atomicMax(bits, (unsigned long long)__double_as_longlong((double)m));
  }
  __syncthreads();  // wmax is reused by the next call of the block
}

// Returns the cell's inverse CFL contribution (0 outside the grid), in the bulk type.
// FP32 bulk converts its 8 FP32 increments to FP64 with one warp vote (ONE_VOTE), or each
// by a select (fewer registers live at once: the batch kernels, which also hold a member's
// header, keep their occupancy that way).
template <typename T, bool COMBINE, bool POT = false, bool ONE_VOTE = true>
__device__ __forceinline__ T update_body(const Geo& g, const Ptr8<const double>& Uin,
                                              const Ptr8<const double>& U0,
                                              const Ptr8<const T>& Fx, const Ptr8<const T>& Fy,
                                              const Ptr8<const T>& Fz, const T* Ex, const T* Ey,
                                              const T* Ez, const Ptr8<double>& Uout, double dt,
                                              int c, double w = 0.5, double w0 = 0.5,
                                              const PotStage* pot = nullptr) {
  T inv = T(0);
  if (c < g.ncell) {
    int ijk[3];
    coords(g, c, ijk[0], ijk[1], ijk[2]);
    const Ptr8<const T> F[3] = {Fx, Fy, Fz};
    const T* E[3] = {Ex, Ey, Ez};
    int up[3];
    upper_offsets(g, ijk, up);
#pragma unroll
    for (int d = 0; d < 3; ++d) up[d] += c;
    // flux divergence and EMF curl in the bulk type T; the accumulation into the
    // state is FP64 in both variants.  FP32 bulk also forms dt * div in FP32 (the
    // increment only needs FP32 precision) and adds it to the FP64 state.
    auto idl = [&](int d) -> T {
      if constexpr (std::is_same<T, double>::value) return g.inv_dl[d];
      else return g.inv_dlf[d];
    };
    // the scaled step is formed once per cell (one FP64 product), not once per field
    [[maybe_unused]] const float dtf =
        std::is_same<T, float>::value ? d2f_warp(COMBINE ? w * dt : dt) : 0.f;
    // FP32 bulk: the FP32 increments -w dt (div) of the 8 fields, converted to FP64 together
    // (one warp vote for the rare subnormal lanes) and then accumulated
    [[maybe_unused]] float finc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    auto accumulate = [&](int f, double dinc) -> double {
      if (COMBINE) {
        if (w == w0) return fma(w, U0.f[f][c] + Uin.f[f][c], dinc);
        return fma(w0, U0.f[f][c], w * Uin.f[f][c]) + dinc;
      }
      return Uin.f[f][c] + dinc;
    };
    // FP64: dt folded into the inverse cell sizes, each difference accumulated by one FMA
    double kdt[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) kdt[d] = dt * g.inv_dl[d];
    double out[8];
#ifdef IDX_STRICT_ROUNDING
    if constexpr (std::is_same<T, double>::value && !POT) {
      // strict-rounding build: differences over the cell size summed from zero, then
      // U - dt (sum) and w U* + w0 U0, each rounded on its own
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        double div = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (!g.active[d]) continue;
          const int s = slot(f, d);
          div = div + (F[d].f[s][up[d]] - F[d].f[s][c]) / g.dl[d];
        }
        out[f] = Uin.f[f][c] - dt * div;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
        double curl = 0.0;
        if (g.active[d]) {
          if (g.active[t1]) curl = curl + (E[t2][up[t1]] - E[t2][c]) / g.dl[t1];
          if (g.active[t2]) curl = curl - (E[t1][up[t2]] - E[t1][c]) / g.dl[t2];
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (a == d || !g.active[a]) continue;
            const int s = slot(5 + d, a);
            curl = curl + (F[a].f[s][up[a]] - F[a].f[s][c]) / g.dl[a];
          }
        }
        out[5 + d] = Uin.f[5 + d][c] - dt * curl;
      }
#pragma unroll
      for (int f = 0; f < 8; ++f) Uout.f[f][c] = COMBINE ? w * out[f] + w0 * U0.f[f][c] : out[f];
      double s = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!g.active[d]) continue;
        const double a = F[d].f[7][c], b = F[d].f[7][up[d]];
        s = s + (a < b ? b : a) / g.dl[d];
      }
      return s;
    }
#endif
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      if constexpr (std::is_same<T, double>::value) {
        double acc = Uin.f[f][c];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (!g.active[d]) continue;
          const int s = slot(f, d);
          acc = fma(F[d].f[s][c] - F[d].f[s][up[d]], kdt[d], acc);
        }
        out[f] = acc;
      } else {
        T div = T(0);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (!g.active[d]) continue;
          const int s = slot(f, d);
          div += (F[d].f[s][up[d]] - F[d].f[s][c]) * idl(d);
        }
        finc[f] = -dtf * div;
      }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      if constexpr (POT) {
        // Eq. 8: the face field is the circulation of the stepped potential
        double b = pot->bref[d][c];
        if (g.active[t1]) b += (pot->out[t2][up[t1]] - pot->out[t2][c]) * g.inv_dl[t1];
        if (g.active[t2]) b -= (pot->out[t1][up[t2]] - pot->out[t1][c]) * g.inv_dl[t2];
        out[5 + d] = b;
        continue;
      }
      if constexpr (std::is_same<T, double>::value) {
        double acc = Uin.f[5 + d][c];
        if (g.active[d]) {
          if (g.active[t1]) acc = fma(E[t2][c] - E[t2][up[t1]], kdt[t1], acc);
          if (g.active[t2]) acc = fma(E[t1][up[t2]] - E[t1][c], kdt[t2], acc);
        } else {
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (a == d || !g.active[a]) continue;
            const int s = slot(5 + d, a);
            acc = fma(F[a].f[s][c] - F[a].f[s][up[a]], kdt[a], acc);
          }
        }
        out[5 + d] = acc;
        continue;
      }
      T curl = T(0);
      if (g.active[d]) {
        if (g.active[t1]) curl += (E[t2][up[t1]] - E[t2][c]) * idl(t1);
        if (g.active[t2]) curl -= (E[t1][up[t2]] - E[t1][c]) * idl(t2);
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a == d || !g.active[a]) continue;
          const int s = slot(5 + d, a);
          curl += (F[a].f[s][up[a]] - F[a].f[s][c]) * idl(a);
        }
      }
      finc[5 + d] = -dtf * curl;
    }
    if constexpr (std::is_same<T, float>::value) {
      double dinc[8];
      if constexpr (ONE_VOTE) {
        f2d_many(finc, dinc);
      } else {
#pragma unroll
        for (int f = 0; f < 8; ++f) dinc[f] = f2d(finc[f]);
      }
#pragma unroll
      for (int f = 0; f < 8; ++f)
        if (!(POT && f >= 5)) out[f] = accumulate(f, dinc[f]);
    }
#pragma unroll
    for (int f = 0; f < 8; ++f)
      Uout.f[f][c] = (COMBINE && std::is_same<T, double>::value && !(POT && f >= 5))
                         ? fma(w, out[f], w0 * U0.f[f][c])
                         : out[f];
    T invT = T(0);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (g.active[d]) invT += max_nn(F[d].f[7][c], F[d].f[7][up[d]]) * idl(d);
    inv = invT;
  }
  return inv;
}

template <typename T, bool COMBINE, bool POT = false>
__global__ void __launch_bounds__(kThreads) k_update(Geo g, Ptr8<const double> Uin,
                                                     Ptr8<const double> U0, Ptr8<const T> Fx,
                                                     Ptr8<const T> Fy, Ptr8<const T> Fz,
                                                     const T* Ex, const T* Ey, const T* Ez,
                                                     Ptr8<double> Uout, Ctrl* ctrl, double w,
                                                     double w0, PotStage pot) {
  const double dt = ctrl->dt;
  if (!(dt > 0.0)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const T inv = update_body<T, COMBINE, POT>(g, Uin, U0, Fx, Fy, Fz, Ex, Ey, Ez, Uout, dt, c, w,
                                             w0, &pot);
  // block max -> one atomic per block (positive doubles order like their bit patterns)
  block_max_to(&ctrl->inv_acc, inv);
}

// FP32 bulk, RK2, field form: the update of a stage that also recovers the primitives of
// the state it forms, for the next stage (or the next cycle), so that the primitive
// recovery reads no state of its own from HBM.  The RK2 combine U^{n+1} = (U^n + U*)/2 +
// (dt/2) L(U*) (Eq. 9) is carried as the half sum S = (U^n + U*)/2 = U^n + (dt/2) L(U^n):
//   stage 1 (STAGE2 false): U* = U^n + dt L(U^n) only in registers, for its primitives;
//                           S -> Uout (all 8 fields), the face fields of U* -> Bs (the
//                           normal field the stage-2 sweeps read);
//   stage 2 (STAGE2 true):  U^{n+1} = S + (dt/2) L(U*) -> Uout, from S alone.
// Each cell forms the stepped fields of its three lower faces and, for the cell-centre B
// of its primitives, of its three upper faces (the lower faces of its upper neighbours,
// formed again there).  The increments are FP32 (as in k_update<float>); every sum into the
// state is FP64.  Stage-2 primitives belong to the next cycle: a non-physical cell there is
// recorded in bad_next, which the next cycle's k_begin turns into the error.
// The kernel is bound by latency and instruction issue more than by its bytes (the same
// loads and stores without the arithmetic run at the copy bandwidth): neighbour offsets
// are formed once per cell, coordinates by multiply-and-shift division, and stage 2 runs
// 6 blocks per SM (40 registers); stage 1, which holds more values, 5.
template <bool STAGE2>
__global__ void __launch_bounds__(kThreads, STAGE2 ? 6 : 5) k_update_carry(Geo g, Ptr8<const double> Uin,
                                                           Ptr8<const float> Fx,
                                                           Ptr8<const float> Fy,
                                                           Ptr8<const float> Fz,
                                                           const float* Ex, const float* Ey,
                                                           const float* Ez, Ptr8<double> Uout,
                                                           Ptr3 Bs, Ptr8<float> W,
                                                           CellEmf<float> cc, Ctrl* ctrl) {
  const double dt = ctrl->dt;
  if (!(dt > 0.0)) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  float inv = 0.f;
  if (c < g.ncell) {
    int ijk[3];
    coords(g, c, ijk[0], ijk[1], ijk[2]);
    const Ptr8<const float> F[3] = {Fx, Fy, Fz};
    const float* E[3] = {Ex, Ey, Ez};
    // offsets of the upper neighbour along each direction (periodic wrap); the cell's edges
    // and faces sit at c plus sums of them
    int off[3], up[3];
    upper_offsets(g, ijk, off);
#pragma unroll
    for (int d = 0; d < 3; ++d) up[d] = c + off[d];
    // stage 1 steps by dt, stage 2 by dt/2 (the RK2 weight of L(U*))
    const float dtf = d2f_warp(STAGE2 ? 0.5 * dt : dt);
    // FP32 increments: the 5 cell fields, then the field normal to d on the lower d-face
    // (5 + d) and on the upper one (8 + d, the lower face of the upper neighbour, whose
    // coordinates along the other two directions are those of c)
    float inc[11];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      float div = 0.f;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (!g.active[d]) continue;
        const int sl = slot(f, d);
        div += (F[d].f[sl][up[d]] - F[d].f[sl][c]) * g.inv_dlf[d];
      }
      inc[f] = -dtf * div;
    }
    auto face_inc = [&](int d, int q) -> float {
      const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
      float curl = 0.f;
      if (g.active[d]) {
        if (g.active[t1]) curl += (E[t2][q + off[t1]] - E[t2][q]) * g.inv_dlf[t1];
        if (g.active[t2]) curl -= (E[t1][q + off[t2]] - E[t1][q]) * g.inv_dlf[t2];
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a == d || !g.active[a]) continue;
          const int sl = slot(5 + d, a);
          curl += (F[a].f[sl][q + off[a]] - F[a].f[sl][q]) * g.inv_dlf[a];
        }
      }
      return -dtf * curl;
    };
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      inc[5 + d] = face_inc(d, c);
      // a one-cell direction: the upper face is the lower one
      inc[8 + d] = g.active[d] ? face_inc(d, up[d]) : inc[5 + d];
    }
    double dinc[11];
    f2d_many(inc, dinc);
    double u[5], b0[3], b1[3];
#pragma unroll
    for (int f = 0; f < 5; ++f) u[f] = Uin.f[f][c] + dinc[f];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      b0[d] = Uin.f[5 + d][c] + dinc[5 + d];
      b1[d] = g.active[d] ? Uin.f[5 + d][up[d]] + dinc[8 + d] : b0[d];
    }
    if (STAGE2) {
#pragma unroll
      for (int f = 0; f < 5; ++f) Uout.f[f][c] = u[f];
#pragma unroll
      for (int d = 0; d < 3; ++d) Uout.f[5 + d][c] = b0[d];
    } else {
      // the half sum S = U^n + inc / 2 (halving the FP64 image of inc: exact)
#pragma unroll
      for (int f = 0; f < 8; ++f) Uout.f[f][c] = Uin.f[f][c] + half_of_f32_image(dinc[f]);
#pragma unroll
      for (int d = 0; d < 3; ++d) Bs.f[d][c] = b0[d];
    }
    if (prims_f32_vals(g, u[0], u[1], u[2], u[3], u[4], b0[0], b1[0], b0[1], b1[1], b0[2],
                       b1[2], W, cc, c)) {
      if (STAGE2) flag_bad_next(ctrl, c);
      else flag_bad(ctrl, c);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (g.active[d]) inv += max_nn(F[d].f[7][c], F[d].f[7][up[d]]) * g.inv_dlf[d];
  }
  block_max_to(&ctrl->inv_acc, inv);
}

// Primitives of the state U for the first cycle of the carried-primitive stages (after
// another path changed the state): a non-physical cell goes to bad_next, as if the last
// cycle's update had found it.
__global__ void __launch_bounds__(kThreads, 6) k_prims_next(Geo g, Ptr8<const double> U,
                                                            Ptr8<float> W, CellEmf<float> cc,
                                                            Ctrl* ctrl) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int i, j, k;
  coords(g, c, i, j, k);
  if (prims_f32_vals(g, U.f[0][c], U.f[1][c], U.f[2][c], U.f[3][c], U.f[4][c], U.f[5][c],
                     U.f[5][shifted(g, c, i, 0, 1)], U.f[6][c], U.f[6][shifted(g, c, j, 1, 1)],
                     U.f[7][c], U.f[7][shifted(g, c, k, 2, 1)], W, cc, c))
    flag_bad_next(ctrl, c);
}

// Inverse CFL time of a state from the face speeds alone (first cycle).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_inv_only(Geo g, Ptr8<const T> Fx, Ptr8<const T> Fy,
                                                       Ptr8<const T> Fz, Ctrl* ctrl) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  double inv = 0.0;
  if (c < g.ncell) {
    int ijk[3];
    coords(g, c, ijk[0], ijk[1], ijk[2]);
    const Ptr8<const T> F[3] = {Fx, Fy, Fz};
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (g.active[d]) {
        const int u = shifted(g, c, ijk[d], d, 1);
#ifdef IDX_STRICT_ROUNDING
        inv = inv + fmax(double(F[d].f[7][c]), double(F[d].f[7][u])) / g.dl[d];
#else
        inv += fmax(double(F[d].f[7][c]), double(F[d].f[7][u])) * g.inv_dl[d];
#endif
      }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) inv = fmax(inv, __shfl_xor_sync(0xffffffffu, inv, o));
  __shared__ double wmax[kThreads / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = inv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = wmax[0];
    for (int w = 1; w < kThreads / 32; ++w) m = fmax(m, wmax[w]);
    atomicMax(&ctrl->inv_prev, (unsigned long long)__double_as_longlong(m));
  }
}

// Cycle prologue: dt = cfl / inv (Eq. 10), clamped to t_end - t.
__device__ __forceinline__ void begin_body(Ctrl* c) {
  if (c->err != 0 || c->done) {
    c->dt = 0.0;
    c->done = 1;
    return;
  }
  const double inv = __longlong_as_double((long long)c->inv_prev);
  double dt = c->cfl / inv;
  const double rem = c->t_end - c->t;
  int clamped = 0;
  if (dt > rem) dt = rem;
  if (dt >= rem) clamped = 1;
  if (!(dt > 0.0)) {
    c->dt = 0.0;
    c->done = 1;
    return;
  }
  c->dt = dt;
  c->clamped = clamped;
  c->inv_acc = 0ull;
  if (c->bad_next != ~0ull) {  // the cycle starts from a non-physical state
    c->err = IDX_ENONPHYS;
    c->bad_cell = c->bad_next < c->bad_cell ? c->bad_next : c->bad_cell;
    c->bad_next = ~0ull;
  }
}

// Cycle epilogue: advance t, keep the larger stage speed bound for the next dt.
__device__ __forceinline__ void end_body(Ctrl* c) {
  if (!(c->dt > 0.0)) return;
  c->t = c->clamped ? c->t_end : c->t + c->dt;
  c->last_dt = c->dt;
  c->inv_prev = c->inv_acc;
  c->nsteps += 1;
  if (c->clamped) c->done = 1;
  c->dt = 0.0;
}

__global__ void k_begin(Ctrl* c) { begin_body(c); }
__global__ void k_end(Ctrl* c) { end_body(c); }

#include "fused_stage.cuh"

}  // namespace

// ===========================================================================
// Host side
// ===========================================================================
struct idx_sim {
  idx_grid grid;
  double gamma;
  idx_solver solver;
  Geo geo;
  cudaStream_t stream;
  bool own_stream;
  int device;
  int nsm = 0;          // SMs of the device (0: not known, full-size blocks)
  // unique per sim in the process: a destroyed sim's host address can come back for a new
  // one, so captured graphs that hold a sim's buffers are matched by serial, not address
  uint64_t serial = 0;
  // small grids: the y and z sweeps of a stage run on two side streams beside the x sweep
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr, join_ev[2] = {nullptr, nullptr};
  void* mem;            // single device allocation
  size_t mem_bytes;
  Ptr8<double> U, U1;   // state and first-stage result (FP64)
  Ptr8<double> U2;      // second-stage result of RK3 (FP64)
  Ptr8<double> Wd, Fd[3];
  Ptr8<float> Wf, Ff[3];
  double* Ed[3];
  float* Ef[3];
  CellEmf<double> Cd;   // cell-centre EMFs (null in the no-allocation path)
  CellEmf<float> Cf;
  bool pot;             // vector-potential induction (Eqs. 7-8)
  Ptr3 A, A1, A2;       // edge potential of the state and of the stage results
  Ptr3 Bref;            // fixed face field: B = Bref + curl A
  int bc[3];            // boundary kind per direction (periodic along a one-cell direction)
  bool bounded;         // some direction is not periodic: the grid is padded
  Ctrl* ctrl;           // device
  Ctrl* host_ctrl;      // pinned mirror
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int64_t last_bad;
  int sweep_shape[3];   // per direction: marching segment (2..32), -1 warp x-sweep,
                        // 100 + L TMA-staged tile of L faces (y, z), 0 default
  CUtensorMap tm_body[3][2];  // per direction (y, z used): box of L = 16 / 32 rows
  CUtensorMap tm_halo[3];     // per direction: box of the 2 halo rows
  bool tma_ok[3][2];          // maps encoded for L = 16 / 32 and nx % 32 == 0
  bool tuned;
  // FP32 bulk: the fused stage kernel (k_stage_fused) in place of the sweeps, E^c and update
  FusedMaps fmaps;            // primitive-plane boxes of its tiles
  bool fused_ok;              // the grid and solver fit it
  int fused_zc;               // z-planes per CTA
  int stage_mode;             // 0 automatic, 1 split kernels, 2 fused kernel, 3 carried
  bool use_fused;             // the choice the captured cycle holds
  // FP32 bulk, RK2, field form, periodic: the updates also recover the next stage's
  // primitives (k_update_carry), so a stage has no primitive-recovery kernel
  bool carry_ok;              // the sim fits it (Bs allocated)
  bool use_carry;             // the choice the captured cycle holds
  bool w_fresh;               // W and the cell-centre EMFs hold the primitives of U
  Ptr3 Bs;                    // stage-1 face fields (the stage-2 sweeps' normal field)
};

namespace {

#define IDX_TRY(x)                                  \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return IDX_ECUDA;        \
  } while (0)

unsigned blocks_for(long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// x sweep: one warp per 32 cells of an x-row
unsigned blocks_x(const Geo& g) {
  const long warps = (long)g.n[1] * g.n[2] * ((g.n[0] + 31) / 32);
  return blocks_for(warps * 32);
}

template <typename T> CellEmf<T> cell_emf(const idx_sim* s);
template <> CellEmf<double> cell_emf<double>(const idx_sim* s) { return s->Cd; }
template <> CellEmf<float> cell_emf<float>(const idx_sim* s) { return s->Cf; }

template <typename T> Ptr8<const T> cst(const Ptr8<T>& p) {
  Ptr8<const T> q;
  for (int f = 0; f < 8; ++f) q.f[f] = p.f[f];
  return q;
}

// Block size of a marching sweep of nthr threads: full blocks, halved (down to one warp)
// while the launch would give fewer than two blocks per SM -- a small grid then spreads
// over the GPU instead of running a few full blocks on a few SMs.
int march_block(const idx_sim* s, long nthr) {
  int nt = kThreads;
  while (s->nsm > 0 && nt > 32 && (nthr + nt - 1) / nt < 2L * s->nsm) nt >>= 1;
  return nt;
}

// One sweep launch in the given shape (see idx_sim::sweep_shape).
template <typename T, int D, int SEG, int RECON = 1>
void launch_march(idx_sim* s, const Ptr8<T>& W, const double* bface, const Ptr8<T>& F,
                  int check_dt) {
  const Geo& g = s->geo;
  const int a = (D + 1) % 3, b = (D + 2) % 3;
  const long nthr = (long)g.n[a] * g.n[b] * ((g.n[D] + SEG - 1) / SEG);
  const int nt = march_block(s, nthr);
  k_sweep<T, D, SEG, RECON><<<(unsigned)((nthr + nt - 1) / nt), nt, 0, s->stream>>>(
      g, cst(W), bface, F, s->ctrl, check_dt);
}

template <typename T, int D, int L, int RECON = 1>
void launch_tma(idx_sim* s, const double* bface, const Ptr8<T>& F, int check_dt) {
  const Geo& g = s->geo;
  const int nO = g.n[D == 1 ? 2 : 1];
  const unsigned blocks = (unsigned)((g.n[0] / 32) * (g.n[D] / L) * nO);
  const size_t smem = 7 * (L + 4) * 32 * sizeof(T);
  k_sweep_tma<T, D, L, RECON><<<blocks, 8 * L, smem, s->stream>>>(
      g, s->tm_body[D][L == 32 ? 1 : 0], s->tm_halo[D], bface, F, s->ctrl, check_dt);
}

// The FP64 tile of 32 rows takes 63 KB of shared memory, above the 48 KB default.
void allow_tma_smem() {
  cudaFuncSetAttribute(k_stage_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused::SMEM_BYTES);
  cudaFuncSetAttribute(k_stage_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused::SMEM_BYTES);
  const int big = 7 * (32 + 4) * 32 * (int)sizeof(double);
  cudaFuncSetAttribute(k_sweep_tma<double, 1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_sweep_tma<double, 2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_sweep_tma<double, 1, 32, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_sweep_tma<double, 2, 32, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaGetLastError();
}

// Shapes a direction can take: 100 + L only where the staged tiles fit the grid.
bool tma_shape_ok(const idx_sim* s, int d, int shape) {
  if (shape == -2) return d == 0 && s->tma_ok[0][0];
  if (shape != 116 && shape != 132) return true;
  return d != 0 && s->tma_ok[d][shape == 132 ? 1 : 0] && s->geo.n[d] % (shape - 100) == 0;
}

template <typename T> void launch_tma_x(idx_sim* s, const Ptr8<T>& W, const double* bface,
                                        const Ptr8<T>& F, int check_dt) {
  const Geo& g = s->geo;
  const unsigned blocks = (unsigned)((g.n[0] / 32) * (g.n[1] / kXRows) * g.n[2]);
  k_sweep_tma_x<T><<<blocks, 32 * kXRows, 0, s->stream>>>(g, s->tm_body[0][0], cst(W), bface,
                                                          F, s->ctrl, check_dt);
}

template <typename T, int D>
void launch_sweep_d(idx_sim* s, int shape, const Ptr8<T>& W, const double* bface,
                    const Ptr8<T>& F, int check_dt) {
  if (s->geo.recon == 3) {  // LimO3: marching sweeps of 16 or 32 faces, staged y/z tiles
    if (D != 0 && tma_shape_ok(s, D, shape)) {
      if (shape == 116) { launch_tma<T, (D == 0 ? 1 : D), 16, 3>(s, bface, F, check_dt); return; }
      if (shape == 132) { launch_tma<T, (D == 0 ? 1 : D), 32, 3>(s, bface, F, check_dt); return; }
    }
    if (shape == 32) launch_march<T, D, 32, 3>(s, W, bface, F, check_dt);
    else launch_march<T, D, 16, 3>(s, W, bface, F, check_dt);
    return;
  }
  if (D == 0 && shape == -2 && tma_shape_ok(s, 0, -2)) {
    launch_tma_x<T>(s, W, bface, F, check_dt);
    return;
  }
  if (D != 0 && tma_shape_ok(s, D, shape)) {
    if (shape == 116) { launch_tma<T, (D == 0 ? 1 : D), 16>(s, bface, F, check_dt); return; }
    if (shape == 132) { launch_tma<T, (D == 0 ? 1 : D), 32>(s, bface, F, check_dt); return; }
  }
  switch (shape) {
    case -1:
      if (D == 0) {
        k_sweep_x<T><<<blocks_x(s->geo), kThreads, 0, s->stream>>>(s->geo, cst(W), bface, F,
                                                                     s->ctrl, check_dt);
        return;
      }
      break;
    case 2: launch_march<T, D, 2>(s, W, bface, F, check_dt); return;
    case 4: launch_march<T, D, 4>(s, W, bface, F, check_dt); return;
    case 8: launch_march<T, D, 8>(s, W, bface, F, check_dt); return;
    case 16: launch_march<T, D, 16>(s, W, bface, F, check_dt); return;
    case 32: launch_march<T, D, 32>(s, W, bface, F, check_dt); return;
    default: break;
  }
  // not tuned: grids below the tuning size take 2-face segments, which give them 8x the
  // threads of the default at one extra cell slope per 2 faces
  if (s->geo.ncell < kTuneMinCells) launch_march<T, D, 2>(s, W, bface, F, check_dt);
  else launch_march<T, D, kSegDefault>(s, W, bface, F, check_dt);
}

template <typename T>
void launch_sweep(idx_sim* s, int d, const Ptr8<T>& W, const double* bface, const Ptr8<T>& F,
                  int check_dt) {
  const int shape = s->sweep_shape[d];
  if (d == 0) launch_sweep_d<T, 0>(s, shape, W, bface, F, check_dt);
  else if (d == 1) launch_sweep_d<T, 1>(s, shape, W, bface, F, check_dt);
  else launch_sweep_d<T, 2>(s, shape, W, bface, F, check_dt);
}

// Autotuner of the sweep shape: per integrated direction, time every candidate shape on
// the sim's current primitives (three launches each, CUDA events, fastest wins).  All
// shapes do the same arithmetic per face (up to the compiler's FMA contractions).
template <typename T>
int tune_sweeps(idx_sim* s, const Ptr8<double>& U, const Ptr8<T>& W, Ptr8<T>* F) {
  const Geo& g = s->geo;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return IDX_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return IDX_ECUDA; }
  const int cand[9] = {-1, -2, 2, 4, 8, 16, 32, 116, 132};
  int rc = IDX_OK;
  for (int d = 0; d < 3 && rc == IDX_OK; ++d) {
    if (!g.active[d]) continue;
    float best = 1e30f;
    int best_shape = kSegDefault;
    for (int q = 0; q < 9; ++q) {
      const int shape = cand[q];
      // LimO3: marching 16 / 32 and the staged y/z tiles
      if (g.recon == 3 && shape != 16 && shape != 32 && shape != 116 && shape != 132) continue;
      if (shape < 0 && d != 0) continue;
      if ((shape > 100 || shape == -2) && !tma_shape_ok(s, d, shape)) continue;
      if (shape > 0 && shape < 100 && shape > 2 * g.n[d]) continue;
      s->sweep_shape[d] = shape;
      launch_sweep<T>(s, d, W, U.f[5 + d], F[d], 0);
      cudaEventRecord(e0, s->stream);
      for (int r = 0; r < 3; ++r) launch_sweep<T>(s, d, W, U.f[5 + d], F[d], 0);
      cudaEventRecord(e1, s->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = IDX_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_shape = shape; }
    }
    s->sweep_shape[d] = best_shape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == IDX_OK && cudaGetLastError() != cudaSuccess) rc = IDX_ECUDA;
  return rc;
}

// The sweeps of a stage, with the normal face field of direction d from bface[d].
template <typename T>
void launch_sweeps(idx_sim* s, const double* const bface[3], const Ptr8<T>& W, Ptr8<T>* F,
                   int check_dt, bool fork) {
  const Geo& g = s->geo;
  if (!(fork && s->side[0])) {
    for (int d = 0; d < 3; ++d)
      if (g.active[d]) launch_sweep<T>(s, d, W, bface[d], F[d], check_dt);
    return;
  }
  // the three sweeps read the primitives and write their own fluxes: y and z on the side
  // streams, forked after the primitives and joined before the EMFs
  const cudaStream_t main = s->stream;
  cudaEventRecord(s->fork_ev, main);
  if (g.active[0]) launch_sweep<T>(s, 0, W, bface[0], F[0], check_dt);
  for (int d = 1; d < 3; ++d) {
    if (!g.active[d]) continue;
    cudaStreamWaitEvent(s->side[d - 1], s->fork_ev, 0);
    s->stream = s->side[d - 1];
    launch_sweep<T>(s, d, W, bface[d], F[d], check_dt);
    s->stream = main;
    cudaEventRecord(s->join_ev[d - 1], s->side[d - 1]);
    cudaStreamWaitEvent(main, s->join_ev[d - 1], 0);
  }
}

template <typename T>
void launch_fluxes(idx_sim* s, const Ptr8<double>& Uin, const Ptr8<T>& W, Ptr8<T>* F,
                   int check_dt, bool fork = false) {
  const Geo& g = s->geo;
  k_prims<T><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(g, cst(Uin), W, cell_emf<T>(s),
                                                              s->ctrl, check_dt);
  const double* const bface[3] = {Uin.f[5], Uin.f[6], Uin.f[7]};
  launch_sweeps<T>(s, bface, W, F, check_dt, fork);
}

// The stages of one cycle (Sec. 2.7, Table 1): input, output and weights (w, w0) of
// U_s = w S_dt(U_{s-1}) + w0 U_0.  RK2: U -> U1 -> U; RK3: U -> U1 -> U2 -> U.  The
// edge potential of the vector-potential form follows the same registers (A, A1, A2).
struct StagePlan {
  int n;
  const Ptr8<double>* in[3];
  const Ptr8<double>* out[3];
  const Ptr3* ain[3];
  const Ptr3* aout[3];
  double w[3], w0[3];
};

StagePlan stage_plan(const idx_sim* s) {
  StagePlan p;
  if (s->solver.rk_order == 3) {
    p.n = 3;
    p.in[0] = &s->U; p.out[0] = &s->U1; p.w[0] = 1.0; p.w0[0] = 0.0;
    p.in[1] = &s->U1; p.out[1] = &s->U2; p.w[1] = 0.25; p.w0[1] = 0.75;
    p.in[2] = &s->U2; p.out[2] = &s->U; p.w[2] = 2.0 / 3.0; p.w0[2] = 1.0 / 3.0;
    p.ain[0] = &s->A; p.aout[0] = &s->A1;
    p.ain[1] = &s->A1; p.aout[1] = &s->A2;
    p.ain[2] = &s->A2; p.aout[2] = &s->A;
  } else {
    p.n = 2;
    p.in[0] = &s->U; p.out[0] = &s->U1; p.w[0] = 1.0; p.w0[0] = 0.0;
    p.in[1] = &s->U1; p.out[1] = &s->U; p.w[1] = 0.5; p.w0[1] = 0.5;
    p.in[2] = p.out[2] = nullptr; p.w[2] = p.w0[2] = 0.0;
    p.ain[0] = &s->A; p.aout[0] = &s->A1;
    p.ain[1] = &s->A1; p.aout[1] = &s->A;
    p.ain[2] = p.aout[2] = nullptr;
  }
  return p;
}

PotStage pot_stage(const idx_sim* s, const StagePlan& p, int st) {
  PotStage P;
  for (int e = 0; e < 3; ++e) {
    P.in[e] = s->pot ? p.ain[st]->f[e] : nullptr;
    P.a0[e] = s->pot ? s->A.f[e] : nullptr;
    P.out[e] = s->pot ? p.aout[st]->f[e] : nullptr;
    P.bref[e] = s->pot ? s->Bref.f[e] : nullptr;
  }
  return P;
}

// Edge EMFs of stage st (field form), or the potential step (vector-potential form).
template <typename T>
void launch_emf(idx_sim* s, const StagePlan& p, int st, const Ptr8<T>& W, Ptr8<T>* F, T** E) {
  const Geo& g = s->geo;
  if (!s->pot) {
    k_emf<T><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(
        g, cst(W), cst(F[0]), cst(F[1]), cst(F[2]), cell_emf<T>(s), E[0], E[1], E[2], s->ctrl);
    return;
  }
  const PotStage P = pot_stage(s, p, st);
  if (st > 0)
    k_emf_pot<T, true><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(
        g, cst(W), cst(F[0]), cst(F[1]), cst(F[2]), cell_emf<T>(s), P, s->ctrl, p.w[st],
        p.w0[st]);
  else
    k_emf_pot<T, false><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(
        g, cst(W), cst(F[0]), cst(F[1]), cst(F[2]), cell_emf<T>(s), P, s->ctrl, p.w[st],
        p.w0[st]);
}

template <typename T, bool COMBINE, bool POT>
void launch_update_k(idx_sim* s, const StagePlan& p, int st, Ptr8<T>* F, T** E) {
  const Geo& g = s->geo;
  k_update<T, COMBINE, POT><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(
      g, cst(*p.in[st]), cst(s->U), cst(F[0]), cst(F[1]), cst(F[2]), E[0], E[1], E[2],
      *p.out[st], s->ctrl, p.w[st], p.w0[st], pot_stage(s, p, st));
}

template <typename T>
void launch_update(idx_sim* s, const StagePlan& p, int st, Ptr8<T>* F, T** E) {
  const bool combine = st > 0;
  if (s->pot) {
    if (combine) launch_update_k<T, true, true>(s, p, st, F, E);
    else launch_update_k<T, false, true>(s, p, st, F, E);
  } else {
    if (combine) launch_update_k<T, true, false>(s, p, st, F, E);
    else launch_update_k<T, false, false>(s, p, st, F, E);
  }
}

// Ghost refill of a padded state, direction by direction.
void launch_fill_ghosts(idx_sim* s, const Ptr8<double>& U) {
  if (!s->bounded) return;
  const Geo& g = s->geo;
  for (int d = 0; d < 3; ++d) {
    if (s->bc[d] == IDX_BC_PERIODIC) continue;
    const long long total = 4ll * g.n[(d + 1) % 3] * g.n[(d + 2) % 3];
    k_fill_ghosts<<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, s->stream>>>(
        g, d, s->bc[d], U);
  }
}

// The fused FP32-bulk stage: primitives (without the cell-centre EMFs, which the fused
// kernel forms from the primitives in shared memory), then one kernel for the rest.
void launch_fused(idx_sim* s, const StagePlan& p, int st, double dt_fixed = 0.0) {
  const Geo& g = s->geo;
  const Ptr8<double>& Uin = *p.in[st];
  const unsigned blocks = (unsigned)((g.n[0] / fused::TX) * (g.n[1] / fused::TY) *
                                     (g.n[2] / s->fused_zc));
  if (st > 0)
    k_stage_fused<true><<<blocks, fused::NT, fused::SMEM_BYTES, s->stream>>>(
        g, s->fmaps, Uin.f[5], Uin.f[6], Uin.f[7], cst(Uin), cst(s->U), *p.out[st], s->ctrl,
        s->fused_zc, p.w[st], p.w0[st], dt_fixed);
  else
    k_stage_fused<false><<<blocks, fused::NT, fused::SMEM_BYTES, s->stream>>>(
        g, s->fmaps, Uin.f[5], Uin.f[6], Uin.f[7], cst(Uin), cst(s->U), *p.out[st], s->ctrl,
        s->fused_zc, p.w[st], p.w0[st], dt_fixed);
}

void launch_prims_only(idx_sim* s, const Ptr8<double>& Uin, int check_dt) {
  const Geo& g = s->geo;
  k_prims<float><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(g, cst(Uin), s->Wf,
                                                                  CellEmf<float>{}, s->ctrl,
                                                                  check_dt);
}

template <typename T>
void launch_stage(idx_sim* s, const StagePlan& p, int st, const Ptr8<T>& W, Ptr8<T>* F, T** E) {
  launch_fill_ghosts(s, *p.in[st]);
  if constexpr (std::is_same<T, float>::value) {
    if (s->use_fused) {
      launch_prims_only(s, *p.in[st], 1);
      launch_fused(s, p, st);
      return;
    }
  }
  launch_fluxes<T>(s, *p.in[st], W, F, 1, true);
  launch_emf<T>(s, p, st, W, F, E);
  launch_update<T>(s, p, st, F, E);
}

// The update of stage st of the carried-primitive cycle.
void launch_update_carry(idx_sim* s, int st) {
  const Geo& g = s->geo;
  if (st == 0)
    k_update_carry<false><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(
        g, cst(s->U), cst(s->Ff[0]), cst(s->Ff[1]), cst(s->Ff[2]), s->Ef[0], s->Ef[1],
        s->Ef[2], s->U1, s->Bs, s->Wf, s->Cf, s->ctrl);
  else
    k_update_carry<true><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(
        g, cst(s->U1), cst(s->Ff[0]), cst(s->Ff[1]), cst(s->Ff[2]), s->Ef[0], s->Ef[1],
        s->Ef[2], s->U, s->Bs, s->Wf, s->Cf, s->ctrl);
}

// Normal face fields the sweeps of stage st read: those of U^n, then those of U*.
void carry_bface(const idx_sim* s, int st, const double* bface[3]) {
  for (int d = 0; d < 3; ++d) bface[d] = st == 0 ? s->U.f[5 + d] : s->Bs.f[d];
}

// Both stages of the carried-primitive cycle: sweeps, E^c, update (which also forms the
// primitives of the state it writes).  W and the cell-centre EMFs hold the primitives of
// U on entry and on exit.
void launch_carry_stages(idx_sim* s) {
  const StagePlan p = stage_plan(s);
  for (int st = 0; st < 2; ++st) {
    const double* bface[3];
    carry_bface(s, st, bface);
    launch_sweeps<float>(s, bface, s->Wf, s->Ff, 1, true);
    launch_emf<float>(s, p, st, s->Wf, s->Ff, s->Ef);
    launch_update_carry(s, st);
  }
}

// Before a carried-primitive cycle on stream st: the primitives of U, unless the last
// thing that changed U left them in W already.
void refresh_carry(idx_sim* s, cudaStream_t st) {
  if (!s->use_carry || s->w_fresh) return;
  const Geo& g = s->geo;
  k_prims_next<<<blocks_for(g.ncell), kThreads, 0, st>>>(g, cst(s->U), s->Wf, s->Cf, s->ctrl);
  s->w_fresh = true;
}

void launch_cycle(idx_sim* s) {
  k_begin<<<1, 1, 0, s->stream>>>(s->ctrl);
  if (s->use_carry) {
    launch_carry_stages(s);
    k_end<<<1, 1, 0, s->stream>>>(s->ctrl);
    return;
  }
  const StagePlan p = stage_plan(s);
  for (int st = 0; st < p.n; ++st) {
    if (s->solver.precision == IDX_FP32_BULK)
      launch_stage<float>(s, p, st, s->Wf, s->Ff, s->Ef);
    else
      launch_stage<double>(s, p, st, s->Wd, s->Fd, s->Ed);
  }
  k_end<<<1, 1, 0, s->stream>>>(s->ctrl);
}

// Sweep shapes already tuned in this process, by grid, precision and device.
struct TuneKey {
  int nx, ny, nz, precision, recon, device;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nz, precision, recon, device) <
           std::tie(o.nx, o.ny, o.nz, o.precision, o.recon, o.device);
  }
};
std::map<TuneKey, std::array<int, 3>> g_tune_cache;
std::mutex g_tune_mutex;

// Tune the sweep shapes of a sim before its first stepping (sims stepped only inside a
// batch never need it).  The tuning sweeps recompute the current state's fluxes into
// scratch; the cycle recomputes everything it reads.
// The fused stage kernel runs only when asked for (idx_set_stage_kernels): it does the
// split kernels' arithmetic bit for bit, but measured 2x slower at 256^3 (4.4 ms against
// 2.2 ms for the sweeps, E^c and update it replaces) -- its halo faces and per-face address
// arithmetic make it instruction-bound at two CTAs per SM.
// The carried-primitive stages are the default where they fit (FP32 bulk, RK2, field
// form, periodic).
void choose_stage_kernels(idx_sim* s) {
  s->use_fused = s->fused_ok && s->stage_mode == 2;
  s->use_carry = s->carry_ok && (s->stage_mode == 0 || s->stage_mode == 3);
}

int tune_once(idx_sim* s) {
  choose_stage_kernels(s);
  if (s->tuned) return IDX_OK;
  s->tuned = true;
  if (s->geo.ncell < kTuneMinCells) return IDX_OK;
  const TuneKey key{s->geo.n[0], s->geo.n[1], s->geo.n[2], s->solver.precision, s->geo.recon,
                   s->device};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      for (int d = 0; d < 3; ++d) s->sweep_shape[d] = it->second[d];
      return IDX_OK;
    }
  }
  int rc;
  if (s->solver.precision == IDX_FP32_BULK) {
    launch_fluxes<float>(s, s->U, s->Wf, s->Ff, 0);
    rc = tune_sweeps<float>(s, s->U, s->Wf, s->Ff);
  } else {
    launch_fluxes<double>(s, s->U, s->Wd, s->Fd, 0);
    rc = tune_sweeps<double>(s, s->U, s->Wd, s->Fd);
  }
  if (rc != IDX_OK) return rc;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = {s->sweep_shape[0], s->sweep_shape[1], s->sweep_shape[2]};
  return IDX_OK;
}

// Grids below this many cells run the y and z sweeps beside the x sweep (launch_fluxes):
// each sweep alone leaves most of the GPU idle there.
constexpr int kForkMaxCells = 1 << 21;

int build_graph(idx_sim* s) {
  if (s->exec) return IDX_OK;
  int trc = tune_once(s);
  if (trc != IDX_OK) return trc;
  if (s->geo.ncell < kForkMaxCells && !s->side[0]) {
    for (int k = 0; k < 2; ++k) {
      IDX_TRY(cudaStreamCreateWithFlags(&s->side[k], cudaStreamNonBlocking));
      IDX_TRY(cudaEventCreateWithFlags(&s->join_ev[k], cudaEventDisableTiming));
    }
    IDX_TRY(cudaEventCreateWithFlags(&s->fork_ev, cudaEventDisableTiming));
  }
  IDX_TRY(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
  launch_cycle(s);
  cudaError_t e = cudaStreamEndCapture(s->stream, &s->graph);
  if (e != cudaSuccess) return IDX_ECUDA;
  IDX_TRY(cudaGraphInstantiate(&s->exec, s->graph, 0));
  return IDX_OK;
}

int sync_ctrl(const idx_sim* s) {
  IDX_TRY(cudaMemcpyAsync(s->host_ctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
  IDX_TRY(cudaStreamSynchronize(s->stream));
  return IDX_OK;
}

// Flat index of a cell of the (possibly padded) grid in the user's layout; a ghost cell
// maps to the interior cell it was filled from along each non-periodic direction.
int64_t user_cell(const idx_sim* s, unsigned long long c) {
  if (!s->bounded) return (int64_t)c;
  const Geo& g = s->geo;
  int ijk[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((unsigned long long)g.n[0] * g.n[1]))};
  const int un[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
  for (int d = 0; d < 3; ++d)
    if (s->bc[d]) ijk[d] = std::min(std::max(ijk[d] - 2, 0), un[d] - 1);
  return ijk[0] + (int64_t)un[0] * (ijk[1] + (int64_t)un[1] * ijk[2]);
}

int pending_error(idx_sim* s) {
  if (s->host_ctrl->err != 0) {
    s->last_bad = user_cell(s, s->host_ctrl->bad_cell);
    return s->host_ctrl->err;
  }
  return IDX_OK;
}

// Signal-speed pass on a state: primitives, each direction's face speeds only, and the
// inverse CFL time into ctrl->inv_prev.
template <typename T>
void launch_speed_pass(idx_sim* s, const Ptr8<double>& U, const Ptr8<T>& W, Ptr8<T>* F) {
  const Geo& g = s->geo;
  k_prims<T><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(g, cst(U), W, cell_emf<T>(s),
                                                              s->ctrl, 0);
  for (int d = 0; d < 3; ++d) {
    if (!g.active[d]) continue;
    const long nthr = (long)g.n[(d + 1) % 3] * g.n[(d + 2) % 3] * ((g.n[d] + 15) / 16);
    const int nt = march_block(s, nthr);
    const unsigned nb = (unsigned)((nthr + nt - 1) / nt);
    if (g.recon == 3) {
      if (d == 0) k_sweep_speeds<T, 0, 3><<<nb, nt, 0, s->stream>>>(g, cst(W), U.f[5], F[0]);
      else if (d == 1) k_sweep_speeds<T, 1, 3><<<nb, nt, 0, s->stream>>>(g, cst(W), U.f[6], F[1]);
      else k_sweep_speeds<T, 2, 3><<<nb, nt, 0, s->stream>>>(g, cst(W), U.f[7], F[2]);
    } else {
      if (d == 0) k_sweep_speeds<T, 0, 1><<<nb, nt, 0, s->stream>>>(g, cst(W), U.f[5], F[0]);
      else if (d == 1) k_sweep_speeds<T, 1, 1><<<nb, nt, 0, s->stream>>>(g, cst(W), U.f[6], F[1]);
      else k_sweep_speeds<T, 2, 1><<<nb, nt, 0, s->stream>>>(g, cst(W), U.f[7], F[2]);
    }
  }
  k_inv_only<T><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(g, cst(F[0]), cst(F[1]),
                                                                 cst(F[2]), s->ctrl);
}

// Reset time/flags and run the signal-speed pass on the current state U.
int after_new_state(idx_sim* s) {
  Ctrl c;
  std::memset(&c, 0, sizeof(c));
  c.t = 0.0;
  c.t_end = std::numeric_limits<double>::infinity();
  c.cfl = s->solver.cfl;
  c.bad_cell = ~0ull;
  c.bad_next = ~0ull;
  IDX_TRY(cudaMemcpyAsync(s->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream));
  // the speed pass of the first cycle
  if (s->solver.precision == IDX_FP32_BULK) launch_speed_pass<float>(s, s->U, s->Wf, s->Ff);
  else launch_speed_pass<double>(s, s->U, s->Wd, s->Fd);
  IDX_TRY(cudaGetLastError());
  s->w_fresh = true;  // the speed pass recovered the primitives of U
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  s->last_bad = -1;
  return pending_error(s);
}

// The carried-primitive stages (k_update_carry): FP32 bulk, RK2, field form, periodic (a
// padded grid refills its ghosts before each stage's primitives).
bool carry_fits(bool f32, bool rk3, bool pot, bool bounded) {
  return f32 && !rk3 && !pot && !bounded;
}

// Device bytes of one sim (the single allocation of idx_create); RK3 adds a state, the
// vector-potential form adds Bref and one edge potential per RK register.
size_t sim_bytes(long long ncell, bool f32, bool rk3 = false, bool pot = false,
                 bool bounded = false) {
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t arr_d = align(sizeof(double) * ncell);
  const size_t arr_t = align((f32 ? sizeof(float) : sizeof(double)) * ncell);
  const size_t pot_arrays = pot ? (rk3 ? 12 : 9) : 0;
  const size_t carry_arrays = carry_fits(f32, rk3, pot, bounded) ? 3 : 0;  // Bs
  return ((rk3 ? 24 : 16) + pot_arrays + carry_arrays) * arr_d + (8 + 24 + 3 + 3) * arr_t +
         align(sizeof(Ctrl));
}

using EncodeTiled = PFN_cuTensorMapEncodeTiled_v12000;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
EncodeTiled tensor_map_encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor maps of the staged y/z sweeps: W seen as a 4D array (x, y, z, variable) with
// the variables' arrays field_stride bytes apart; boxes of 32 x-cells by 16, 32 or 2
// rows along the sweep direction, one variable deep.  Host-only encoding.
void encode_sweep_maps(idx_sim* s, void* wbase, size_t elem, size_t field_stride) {
  const Geo& g = s->geo;
  for (int d = 0; d < 3; ++d) s->tma_ok[d][0] = s->tma_ok[d][1] = false;
  if (g.n[0] % 32 != 0) return;
  EncodeTiled enc = tensor_map_encoder();
  if (!enc) return;
  const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], 8};
  const cuuint64_t strides[3] = {(cuuint64_t)g.n[0] * elem, (cuuint64_t)g.n[0] * g.n[1] * elem,
                                 (cuuint64_t)field_stride};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt =
      elem == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  // x: rows of 40 cells (32 and a 4-cell halo on each side), 8 rows deep; the parts
  // past the ends of a row are filled with zeros
  if (g.active[0] && g.n[1] % kXRows == 0) {
    const cuuint32_t box[4] = {(cuuint32_t)kXBox, (cuuint32_t)kXRows, 1, 1};
    s->tma_ok[0][0] = enc(&s->tm_body[0][0], dt, 4, wbase, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  for (int d = 1; d <= 2; ++d) {
    if (!g.active[d]) continue;
    auto encode = [&](unsigned rows, CUtensorMap* m) {
      if ((int)rows > g.n[d]) return false;
      cuuint32_t box[4] = {32, 1, 1, 1};
      box[d] = rows;
      return enc(m, dt, 4, wbase, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                 CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    const bool halo = encode(2, &s->tm_halo[d]);
    s->tma_ok[d][0] = halo && encode(16, &s->tm_body[d][0]);
    s->tma_ok[d][1] = halo && encode(32, &s->tm_body[d][1]);
  }
}

// The fused FP32-bulk stage: fits every-direction-integrated PLM field-form grids with
// nx % 32 == 0 and ny % 8 == 0 (padded grids included: their ghosts are refilled before
// the stage), with a z-chunk that divides nz.  The chunk is the longest of 32, 16, 8, 4, 2
// that still gives every SM two CTAs, so small grids trade some recomputation for work.
void encode_fused_maps(idx_sim* s, void* wbase, size_t field_stride) {
  const Geo& g = s->geo;
  s->fused_ok = false;
  s->fused_zc = 0;
  if (s->solver.recon != 1 || s->pot || !g.active[0] || !g.active[1] || !g.active[2]) return;
  if (g.n[0] % fused::TX != 0 || g.n[1] % fused::TY != 0) return;
  const long tiles_xy = (long)(g.n[0] / fused::TX) * (g.n[1] / fused::TY);
  int zc = 0;
  for (const int c : {32, 16, 8, 4, 2}) {
    if (g.n[2] % c != 0) continue;
    zc = c;
    if (tiles_xy * (g.n[2] / c) >= 2L * (s->nsm > 0 ? s->nsm : 148)) break;
  }
  if (zc == 0) return;
  EncodeTiled enc = tensor_map_encoder();
  if (!enc) return;
  const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], 8};
  const cuuint64_t strides[3] = {(cuuint64_t)g.n[0] * sizeof(float),
                                 (cuuint64_t)g.n[0] * g.n[1] * sizeof(float),
                                 (cuuint64_t)field_stride};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const cuuint32_t bx[2] = {4, (cuuint32_t)fused::TX}, by[2] = {2, (cuuint32_t)fused::TY};
  for (int m = 0; m < 4; ++m) {
    const cuuint32_t box[4] = {bx[m & 1], by[m >> 1], 1, 8};
    if (enc(&s->fmaps.box[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, wbase, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return;
  }
  s->fused_zc = zc;
  s->fused_ok = true;
}

// Boundary kinds of a grid (periodic along a one-cell direction) and the padded cell
// counts; false for an unknown kind or a non-periodic direction of fewer than 2 cells.
bool grid_bc(const idx_grid* grid, int bc[3], int pn[3]) {
  const int n[3] = {grid->nx, grid->ny, grid->nz};
  for (int d = 0; d < 3; ++d) {
    const int k = grid->bc[d];
    if (k != IDX_BC_PERIODIC && k != IDX_BC_OUTFLOW && k != IDX_BC_REFLECTING) return false;
    bc[d] = n[d] > 1 ? k : IDX_BC_PERIODIC;
    pn[d] = n[d] + (bc[d] ? 4 : 0);
  }
  return true;
}

bool valid_solver(const idx_solver* v) {
  return v && (v->recon == 1 || v->recon == 3) &&
         (v->riemann == 1 || v->riemann == 2 || v->riemann == 4) &&
         v->emf == 2 && (v->rk_order == 2 || v->rk_order == 3) &&
         (v->induction == IDX_INDUCTION_FIELD || v->induction == IDX_INDUCTION_POTENTIAL) &&
         v->cfl > 0.0 && v->cfl < 1.0 &&
         (v->precision == IDX_FP64 || v->precision == IDX_FP32_BULK);
}

}  // namespace

extern "C" {

const char* idx_strerror(int code) {
  switch (code) {
    case IDX_OK: return "ok";
    case IDX_EINVAL: return "invalid argument";
    case IDX_ENOMEM: return "device allocation failed";
    case IDX_ENONPHYS: return "non-physical state (rho <= 0, P <= 0 or non-finite)";
    case IDX_ECUDA: return "CUDA runtime error";
    case IDX_ETIMEOUT: return "bounded wait expired";
    case IDX_ETOOLARGE: return "grid larger than the fixed scratch of idx_step_noalloc";
    default: return "unknown error";
  }
}

int idx_create(const idx_grid* grid, double gamma, const idx_solver* solver, void* stream,
               idx_sim** out) {
  if (!out) return IDX_EINVAL;
  *out = nullptr;
  if (!grid || !valid_solver(solver) || !(gamma > 1.0) || !std::isfinite(gamma)) return IDX_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return IDX_EINVAL;
  if (!(grid->lx > 0) || !(grid->ly > 0) || !(grid->lz > 0)) return IDX_EINVAL;
  int bc[3], pn[3];
  if (!grid_bc(grid, bc, pn)) return IDX_EINVAL;
  const bool bounded = bc[0] || bc[1] || bc[2];
  if (bounded && solver->induction == IDX_INDUCTION_POTENTIAL) return IDX_EINVAL;
  const long long ncell = (long long)pn[0] * pn[1] * pn[2];
  if (ncell >= (1ll << 31)) return IDX_EINVAL;

  idx_sim* s = new idx_sim();
  std::memset(s, 0, sizeof(*s));
  s->grid = *grid;
  s->gamma = gamma;
  s->solver = *solver;
  s->last_bad = -1;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return IDX_ECUDA; }
  {
    static std::atomic<uint64_t> next_serial{1};
    s->serial = next_serial.fetch_add(1);
  }
  if (cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess)
    s->nsm = 0;
  for (int d = 0; d < 3; ++d) s->bc[d] = bc[d];
  s->bounded = bounded;
  Geo& g = s->geo;  // the padded grid along non-periodic directions
  g.n[0] = pn[0]; g.n[1] = pn[1]; g.n[2] = pn[2];
  g.stride[0] = 1; g.stride[1] = pn[0]; g.stride[2] = pn[0] * pn[1];
  g.ncell = (int)ncell;
  geo_set_divisors(g);
  const double l[3] = {grid->lx, grid->ly, grid->lz};
  const int un[3] = {grid->nx, grid->ny, grid->nz};
  for (int d = 0; d < 3; ++d) {
    g.active[d] = g.n[d] > 1;
    g.inv_dl[d] = (double)un[d] / l[d];
    g.dl[d] = l[d] / (double)un[d];
    g.inv_dlf[d] = (float)g.inv_dl[d];
  }
  geo_set_gamma(g, gamma);
  g.riemann = solver->riemann;
  g.recon = solver->recon;

  // memory plan: U, U1 (16 doubles/cell) + W, F (3 x 8), E (3) in the bulk type
  const bool f32 = solver->precision == IDX_FP32_BULK;
  const size_t tsz = f32 ? sizeof(float) : sizeof(double);
  auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t arr_d = align(sizeof(double) * ncell), arr_t = align(tsz * ncell);
  const bool rk3 = solver->rk_order == 3;
  s->pot = solver->induction == IDX_INDUCTION_POTENTIAL;
  const size_t bytes = sim_bytes(ncell, f32, rk3, s->pot, bounded);
  if (stream) {
    s->stream = (cudaStream_t)stream;
    s->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return IDX_ECUDA;
    }
    s->own_stream = true;
  }
  // stream-ordered allocation: creating and freeing sims does not synchronise the device
  if (cudaMallocAsync(&s->mem, bytes, s->stream) != cudaSuccess) {
    cudaGetLastError();
    s->mem = nullptr;
    idx_destroy(s);
    return IDX_ENOMEM;
  }
  s->mem_bytes = bytes;
  char* p = (char*)s->mem;
  for (int f = 0; f < 8; ++f) { s->U.f[f] = (double*)p; p += arr_d; }
  for (int f = 0; f < 8; ++f) { s->U1.f[f] = (double*)p; p += arr_d; }
  if (rk3)
    for (int f = 0; f < 8; ++f) { s->U2.f[f] = (double*)p; p += arr_d; }
  s->carry_ok = carry_fits(f32, rk3, s->pot, bounded);
  if (s->carry_ok)
    for (int d = 0; d < 3; ++d) { s->Bs.f[d] = (double*)p; p += arr_d; }
  if (s->pot) {
    for (int e = 0; e < 3; ++e) { s->Bref.f[e] = (double*)p; p += arr_d; }
    for (int e = 0; e < 3; ++e) { s->A.f[e] = (double*)p; p += arr_d; }
    for (int e = 0; e < 3; ++e) { s->A1.f[e] = (double*)p; p += arr_d; }
    if (rk3)
      for (int e = 0; e < 3; ++e) { s->A2.f[e] = (double*)p; p += arr_d; }
  }
  if (f32) {
    for (int f = 0; f < 8; ++f) { s->Wf.f[f] = (float*)p; p += arr_t; }
    for (int d = 0; d < 3; ++d)
      for (int f = 0; f < 8; ++f) { s->Ff[d].f[f] = (float*)p; p += arr_t; }
    for (int d = 0; d < 3; ++d) { s->Ef[d] = (float*)p; p += arr_t; }
    for (int e = 0; e < 3; ++e) { s->Cf.f[e] = (float*)p; p += arr_t; }
  } else {
    for (int f = 0; f < 8; ++f) { s->Wd.f[f] = (double*)p; p += arr_t; }
    for (int d = 0; d < 3; ++d)
      for (int f = 0; f < 8; ++f) { s->Fd[d].f[f] = (double*)p; p += arr_t; }
    for (int d = 0; d < 3; ++d) { s->Ed[d] = (double*)p; p += arr_t; }
    for (int e = 0; e < 3; ++e) { s->Cd.f[e] = (double*)p; p += arr_t; }
  }
  s->ctrl = (Ctrl*)p;
  if (f32) encode_sweep_maps(s, s->Wf.f[0], sizeof(float), arr_t);
  else encode_sweep_maps(s, s->Wd.f[0], sizeof(double), arr_t);
  if (f32) encode_fused_maps(s, s->Wf.f[0], arr_t);
  allow_tma_smem();
  int rc = IDX_OK;
  if (cudaMallocHost(&s->host_ctrl, sizeof(Ctrl)) != cudaSuccess) rc = IDX_ENOMEM;
  // clear on the sim's own stream: a non-blocking stream is not ordered after work
  // on the legacy default stream, so a plain cudaMemset could race the first upload
  if (rc == IDX_OK && cudaMemsetAsync(s->mem, 0, bytes, s->stream) != cudaSuccess) rc = IDX_ECUDA;
  if (rc == IDX_OK && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = IDX_ECUDA;
  if (rc != IDX_OK) {
    idx_destroy(s);
    return rc;
  }
  *out = s;
  return IDX_OK;
}

void idx_destroy(idx_sim* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->host_ctrl) cudaFreeHost(s->host_ctrl);
  if (s->mem) {
    cudaFreeAsync(s->mem, s->stream);
    cudaStreamSynchronize(s->stream);
  }
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  for (int k = 0; k < 2; ++k) {
    if (s->side[k]) cudaStreamDestroy(s->side[k]);
    if (s->join_ev[k]) cudaEventDestroy(s->join_ev[k]);
  }
  if (s->fork_ev) cudaEventDestroy(s->fork_ev);
  delete s;
}

static int copy_fields_in(idx_sim* s, Ptr8<double> dst, const double* const fields[8],
                          int on_device) {
  for (int f = 0; f < 8; ++f)
    if (!fields[f]) return IDX_EINVAL;
  const size_t bytes = sizeof(double) * (size_t)s->geo.ncell;
  for (int f = 0; f < 8; ++f)
    IDX_TRY(cudaMemcpyAsync(dst.f[f], fields[f], bytes,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            s->stream));
  return IDX_OK;
}

// Vector-potential form, state given by its face field: the gauge starts here, A = 0
// and Bref = the face field of U.
static int potential_from_field(idx_sim* s) {
  if (!s->pot) return IDX_OK;
  const size_t bytes = sizeof(double) * (size_t)s->geo.ncell;
  for (int e = 0; e < 3; ++e) {
    IDX_TRY(cudaMemcpyAsync(s->Bref.f[e], s->U.f[5 + e], bytes, cudaMemcpyDeviceToDevice,
                            s->stream));
    IDX_TRY(cudaMemsetAsync(s->A.f[e], 0, bytes, s->stream));
  }
  return IDX_OK;
}

// Padded sims: the user layout of field f (cells, or n + 1 normal faces along a
// non-periodic direction), as a pad descriptor and per-field element counts.
static Pad pad_of(const idx_sim* s, size_t count[8]) {
  Pad pd;
  const int un[3] = {s->grid.nx, s->grid.ny, s->grid.nz};
  for (int d = 0; d < 3; ++d) {
    pd.un[d] = un[d];
    pd.off[d] = s->bc[d] ? 2 : 0;
    pd.ext[d] = s->bc[d] ? 1 : 0;
  }
  for (int f = 0; f < 8; ++f) {
    size_t c = 1;
    for (int d = 0; d < 3; ++d) c *= (size_t)(un[d] + (f == 5 + d ? pd.ext[d] : 0));
    count[f] = c;
  }
  return pd;
}

static unsigned pad_blocks(const Pad& pd) {
  const long long t = (long long)(pd.un[0] + pd.ext[0]) * (pd.un[1] + pd.ext[1]) *
                      (pd.un[2] + pd.ext[2]);
  return (unsigned)((t + kThreads - 1) / kThreads);
}

// User fields (host or device) into the interior of a padded state.  Host fields pass
// through a stream-ordered device staging buffer.
static int pad_in(idx_sim* s, const double* const fields[8], int on_device, Ptr8<double> dst) {
  size_t count[8], total = 0;
  const Pad pd = pad_of(s, count);
  for (int f = 0; f < 8; ++f) total += count[f];
  Ptr8<const double> src;
  double* staging = nullptr;
  if (on_device) {
    for (int f = 0; f < 8; ++f) src.f[f] = fields[f];
  } else {
    if (cudaMallocAsync(&staging, sizeof(double) * total, s->stream) != cudaSuccess) {
      cudaGetLastError();
      return IDX_ENOMEM;
    }
    double* q = staging;
    for (int f = 0; f < 8; ++f) {
      IDX_TRY(cudaMemcpyAsync(q, fields[f], sizeof(double) * count[f], cudaMemcpyHostToDevice,
                              s->stream));
      src.f[f] = q;
      q += count[f];
    }
  }
  k_pad<<<pad_blocks(pd), kThreads, 0, s->stream>>>(s->geo, pd, src, dst, 0);
  IDX_TRY(cudaGetLastError());
  if (staging) IDX_TRY(cudaFreeAsync(staging, s->stream));
  return IDX_OK;
}

// The interior of the padded state U out to user fields (host or device).
static int pad_out(idx_sim* s, double* const fields[8], int on_device) {
  size_t count[8], total = 0;
  const Pad pd = pad_of(s, count);
  for (int f = 0; f < 8; ++f) total += count[f];
  Ptr8<double> dst;
  double* staging = nullptr;
  if (on_device) {
    for (int f = 0; f < 8; ++f) dst.f[f] = fields[f];
  } else {
    if (cudaMallocAsync(&staging, sizeof(double) * total, s->stream) != cudaSuccess) {
      cudaGetLastError();
      return IDX_ENOMEM;
    }
    double* q = staging;
    for (int f = 0; f < 8; ++f) { dst.f[f] = q; q += count[f]; }
  }
  k_pad<<<pad_blocks(pd), kThreads, 0, s->stream>>>(s->geo, pd, cst(s->U), dst, 1);
  IDX_TRY(cudaGetLastError());
  if (staging) {
    for (int f = 0; f < 8; ++f)
      IDX_TRY(cudaMemcpyAsync(fields[f], dst.f[f], sizeof(double) * count[f],
                              cudaMemcpyDeviceToHost, s->stream));
    IDX_TRY(cudaFreeAsync(staging, s->stream));
  }
  return IDX_OK;
}

int idx_set_state(idx_sim* s, const double* const fields[8], int on_device) {
  if (!s || !fields) return IDX_EINVAL;
  if (s->bounded) {
    for (int f = 0; f < 8; ++f)
      if (!fields[f]) return IDX_EINVAL;
    int rc = pad_in(s, fields, on_device, s->U);
    if (rc != IDX_OK) return rc;
    launch_fill_ghosts(s, s->U);
    IDX_TRY(cudaGetLastError());
    return after_new_state(s);
  }
  int rc = copy_fields_in(s, s->U, fields, on_device);
  if (rc == IDX_OK) rc = potential_from_field(s);
  if (rc != IDX_OK) return rc;
  return after_new_state(s);
}

int idx_set_primitive(idx_sim* s, const double* const fields[8], int on_device) {
  if (!s || !fields) return IDX_EINVAL;
  if (s->bounded) {
    // primitives padded into U1 (scratch here), ghosts filled (the velocity flips like the
    // momentum), converted into U, whose ghosts are filled again
    for (int f = 0; f < 8; ++f)
      if (!fields[f]) return IDX_EINVAL;
    int rc = pad_in(s, fields, on_device, s->U1);
    if (rc != IDX_OK) return rc;
    launch_fill_ghosts(s, s->U1);
    k_cons_from_prims<<<blocks_for(s->geo.ncell), kThreads, 0, s->stream>>>(s->geo, cst(s->U1), s->U);
    launch_fill_ghosts(s, s->U);
    IDX_TRY(cudaGetLastError());
    return after_new_state(s);
  }
  // stage the primitives in U1 (scratch at this point), convert into U
  int rc = copy_fields_in(s, s->U1, fields, on_device);
  if (rc != IDX_OK) return rc;
  k_cons_from_prims<<<blocks_for(s->geo.ncell), kThreads, 0, s->stream>>>(s->geo, cst(s->U1), s->U);
  IDX_TRY(cudaGetLastError());
  rc = potential_from_field(s);
  if (rc != IDX_OK) return rc;
  return after_new_state(s);
}

int idx_set_potential(idx_sim* s, const double* const fields[8], const double bmean[3],
                      int on_device) {
  if (!s || !fields || !bmean || s->bounded) return IDX_EINVAL;
  for (int f = 0; f < 8; ++f)
    if (!fields[f]) return IDX_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(bmean[d])) return IDX_EINVAL;
  const size_t bytes = sizeof(double) * (size_t)s->geo.ncell;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // cells staged in U1; the potential goes to A (vector-potential form) or, when it
  // only shapes the initial field, to the face slots of U, which k_cons_from_prims
  // overwrites after k_b_from_pot has read them
  Ptr3 A;
  for (int e = 0; e < 3; ++e) A.f[e] = s->pot ? s->A.f[e] : s->U.f[5 + e];
  for (int f = 0; f < 5; ++f)
    IDX_TRY(cudaMemcpyAsync(s->U1.f[f], fields[f], bytes, kind, s->stream));
  for (int e = 0; e < 3; ++e)
    IDX_TRY(cudaMemcpyAsync(A.f[e], fields[5 + e], bytes, kind, s->stream));
  Vec3 b0;
  for (int d = 0; d < 3; ++d) b0.v[d] = bmean[d];
  Ptr3 B;
  for (int d = 0; d < 3; ++d) B.f[d] = s->U1.f[5 + d];
  k_b_from_pot<<<blocks_for(s->geo.ncell), kThreads, 0, s->stream>>>(s->geo, A, b0, B, s->Bref,
                                                                    s->pot ? 1 : 0);
  k_cons_from_prims<<<blocks_for(s->geo.ncell), kThreads, 0, s->stream>>>(s->geo, cst(s->U1), s->U);
  IDX_TRY(cudaGetLastError());
  return after_new_state(s);
}

int idx_get_potential(const idx_sim* cs, double* const A[3], int on_device) {
  idx_sim* s = const_cast<idx_sim*>(cs);
  if (!s || !A || !s->pot) return IDX_EINVAL;
  for (int e = 0; e < 3; ++e)
    if (!A[e]) return IDX_EINVAL;
  const size_t bytes = sizeof(double) * (size_t)s->geo.ncell;
  for (int e = 0; e < 3; ++e)
    IDX_TRY(cudaMemcpyAsync(A[e], s->A.f[e], bytes,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s->stream));
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  return pending_error(s);
}

int idx_get_state(const idx_sim* cs, double* const fields[8], int on_device) {
  idx_sim* s = const_cast<idx_sim*>(cs);
  if (!s || !fields) return IDX_EINVAL;
  for (int f = 0; f < 8; ++f)
    if (!fields[f]) return IDX_EINVAL;
  if (s->bounded) {
    int rc = pad_out(s, fields, on_device);
    if (rc != IDX_OK) return rc;
    rc = sync_ctrl(s);
    if (rc != IDX_OK) return rc;
    return pending_error(s);
  }
  const size_t bytes = sizeof(double) * (size_t)s->geo.ncell;
  for (int f = 0; f < 8; ++f)
    IDX_TRY(cudaMemcpyAsync(fields[f], s->U.f[f], bytes,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            s->stream));
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  return pending_error(s);
}

int idx_step(idx_sim* s, double* dt_taken) {
  if (!s) return IDX_EINVAL;
  int rc = build_graph(s);
  if (rc != IDX_OK) return rc;
  refresh_carry(s, s->stream);
  IDX_TRY(cudaGraphLaunch(s->exec, s->stream));
  if (!s->use_carry) s->w_fresh = false;
  if (!dt_taken) return IDX_OK;
  rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  rc = pending_error(s);
  if (rc != IDX_OK) return rc;
  *dt_taken = s->host_ctrl->last_dt;
  return IDX_OK;
}

int idx_advance(idx_sim* s, double t_end, int64_t* nsteps) {
  if (!s || !(t_end >= 0.0) || !std::isfinite(t_end)) return IDX_EINVAL;
  int rc = build_graph(s);
  if (rc != IDX_OK) return rc;
  rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  rc = pending_error(s);
  if (rc != IDX_OK) return rc;
  const long long n0 = s->host_ctrl->nsteps;
  // arm the end time
  Ctrl c = *s->host_ctrl;
  c.t_end = t_end;
  c.done = (c.t >= t_end) ? 1 : 0;
  IDX_TRY(cudaMemcpyAsync(s->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream));
  // Graph replays between host checks: the cycles left at the current dt, plus one for the
  // clamped last cycle (at most 256).  Cycles launched past the end exit at once (the
  // device clamps and flags the end), so a growing dt only wastes empty launches and a
  // shrinking one costs another round.
  auto chunk_for = [&](const Ctrl& h) {
    double inv;
    std::memcpy(&inv, &h.inv_prev, sizeof(double));
    const double left = (t_end - h.t) * inv / s->solver.cfl;
    if (!(left >= 0.0) || !(left < 256.0)) return 256;
    return std::max(1, (int)std::ceil(left) + 1);
  };
  int chunk = chunk_for(c);
  refresh_carry(s, s->stream);
  if (!s->use_carry) s->w_fresh = false;
  while (true) {
    for (int q = 0; q < chunk; ++q) IDX_TRY(cudaGraphLaunch(s->exec, s->stream));
    rc = sync_ctrl(s);
    if (rc != IDX_OK) return rc;
    if (s->host_ctrl->err) break;
    if (s->host_ctrl->done) break;
    chunk = chunk_for(*s->host_ctrl);
  }
  // disarm: later idx_step calls run unclamped
  c = *s->host_ctrl;
  c.t_end = std::numeric_limits<double>::infinity();
  c.done = 0;
  IDX_TRY(cudaMemcpyAsync(s->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream));
  IDX_TRY(cudaStreamSynchronize(s->stream));
  if (nsteps) *nsteps = (int64_t)(c.nsteps - n0);
  return pending_error(s);
}

int idx_time(const idx_sim* cs, double* t, double* next_dt) {
  idx_sim* s = const_cast<idx_sim*>(cs);
  if (!s) return IDX_EINVAL;
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  if (t) *t = s->host_ctrl->t;
  if (next_dt) {
    double inv;
    std::memcpy(&inv, &s->host_ctrl->inv_prev, sizeof(double));
    *next_dt = s->solver.cfl / inv;
  }
  return pending_error(s);
}

int idx_kernel_times(idx_sim* s, int reps, double ms[6]) {
  if (!s || !ms || reps < 1) return IDX_EINVAL;
  int rc = tune_once(s);
  if (rc != IDX_OK) return rc;
  rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  rc = pending_error(s);
  if (rc != IDX_OK) return rc;
  cudaEvent_t ev[7];
  for (int q = 0; q < 7; ++q) IDX_TRY(cudaEventCreate(&ev[q]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  int n_stage = 0;
  const Geo& g = s->geo;
  const bool f32 = s->solver.precision == IDX_FP32_BULK;
  refresh_carry(s, s->stream);
  if (!s->use_carry) s->w_fresh = false;
  for (int r = 0; r < reps; ++r) {
    k_begin<<<1, 1, 0, s->stream>>>(s->ctrl);
    const StagePlan plan = stage_plan(s);
    for (int st = 0; st < plan.n; ++st) {
      const Ptr8<double>& Uin = *plan.in[st];
      launch_fill_ghosts(s, Uin);
      IDX_TRY(cudaEventRecord(ev[0], s->stream));
      if (s->use_carry) {
        // carried primitives: no primitive kernel (ms[0] = 0), the update forms them
        IDX_TRY(cudaEventRecord(ev[1], s->stream));
        const double* bface[3];
        carry_bface(s, st, bface);
        for (int d = 0; d < 3; ++d) {
          if (g.active[d]) launch_sweep<float>(s, d, s->Wf, bface[d], s->Ff[d], 1);
          IDX_TRY(cudaEventRecord(ev[2 + d], s->stream));
        }
        launch_emf<float>(s, plan, st, s->Wf, s->Ff, s->Ef);
        IDX_TRY(cudaEventRecord(ev[5], s->stream));
        launch_update_carry(s, st);
        IDX_TRY(cudaEventRecord(ev[6], s->stream));
        IDX_TRY(cudaEventSynchronize(ev[6]));
        float t[6];
        for (int q = 0; q < 6; ++q) IDX_TRY(cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]));
        for (int q = 0; q < 6; ++q) acc[q] += t[q];
        ++n_stage;
        continue;
      }
      if (f32 && s->use_fused) {
        // fused stage: primitives in ms[0], the fused kernel in ms[5], nothing in between
        launch_prims_only(s, Uin, 1);
        for (int q = 1; q <= 5; ++q) IDX_TRY(cudaEventRecord(ev[q], s->stream));
        launch_fused(s, plan, st);
        IDX_TRY(cudaEventRecord(ev[6], s->stream));
        IDX_TRY(cudaEventSynchronize(ev[6]));
        float t[6];
        for (int q = 0; q < 6; ++q) IDX_TRY(cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]));
        for (int q = 0; q < 6; ++q) acc[q] += t[q];
        ++n_stage;
        continue;
      }
      if (f32) {
        k_prims<float><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(g, cst(Uin), s->Wf, s->Cf, s->ctrl, 1);
      } else {
        k_prims<double><<<blocks_for(g.ncell), kThreads, 0, s->stream>>>(g, cst(Uin), s->Wd, s->Cd, s->ctrl, 1);
      }
      IDX_TRY(cudaEventRecord(ev[1], s->stream));
      for (int d = 0; d < 3; ++d) {
        if (g.active[d]) {
          if (f32) launch_sweep<float>(s, d, s->Wf, Uin.f[5 + d], s->Ff[d], 1);
          else launch_sweep<double>(s, d, s->Wd, Uin.f[5 + d], s->Fd[d], 1);
        }
        IDX_TRY(cudaEventRecord(ev[2 + d], s->stream));
      }
      if (f32) launch_emf<float>(s, plan, st, s->Wf, s->Ff, s->Ef);
      else launch_emf<double>(s, plan, st, s->Wd, s->Fd, s->Ed);
      IDX_TRY(cudaEventRecord(ev[5], s->stream));
      if (f32) launch_update<float>(s, plan, st, s->Ff, s->Ef);
      else launch_update<double>(s, plan, st, s->Fd, s->Ed);
      IDX_TRY(cudaEventRecord(ev[6], s->stream));
      IDX_TRY(cudaEventSynchronize(ev[6]));
      float t[6];
      for (int q = 0; q < 6; ++q) IDX_TRY(cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]));
      for (int q = 0; q < 6; ++q) acc[q] += t[q];
      ++n_stage;
    }
    k_end<<<1, 1, 0, s->stream>>>(s->ctrl);
  }
  IDX_TRY(cudaGetLastError());
  for (int q = 0; q < 7; ++q) cudaEventDestroy(ev[q]);
  for (int q = 0; q < 6; ++q) ms[q] = acc[q] / n_stage;
  rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  return pending_error(s);
}

int idx_sweep_shapes(const idx_sim* s, int shapes[3]) {
  if (!s || !shapes) return IDX_EINVAL;
  for (int d = 0; d < 3; ++d) {
    const int v = s->sweep_shape[d];
    const int dflt = (s->geo.recon == 1 && s->geo.ncell < kTuneMinCells) ? 2 : kSegDefault;
    shapes[d] = s->geo.active[d] ? (v == 0 ? dflt : v) : 0;
  }
  return IDX_OK;
}

int idx_set_sweep_shapes(idx_sim* s, const int shapes[3]) {
  if (!s || !shapes) return IDX_EINVAL;
  const Geo& g = s->geo;
  int v[3];
  for (int d = 0; d < 3; ++d) {
    v[d] = g.active[d] ? shapes[d] : 0;
    if (!g.active[d]) continue;
    const int x = v[d];
    if (g.recon == 3) {  // LimO3: marching sweeps of 16 or 32 faces, staged y/z tiles
      const bool ok = x == 16 || x == 32 || ((x == 116 || x == 132) && tma_shape_ok(s, d, x));
      if (!ok) return IDX_EINVAL;
      continue;
    }
    const bool march = x == 2 || x == 4 || x == 8 || x == 16 || x == 32;
    const bool warpx = x == -1 && d == 0;
    const bool staged = (x == 116 || x == 132 || x == -2) && tma_shape_ok(s, d, x);
    if (!march && !warpx && !staged) return IDX_EINVAL;
  }
  for (int d = 0; d < 3; ++d) s->sweep_shape[d] = v[d];
  s->tuned = true;
  // the captured cycle holds the old shapes
  if (s->exec) { cudaGraphExecDestroy(s->exec); s->exec = nullptr; }
  if (s->graph) { cudaGraphDestroy(s->graph); s->graph = nullptr; }
  return IDX_OK;
}

int idx_set_stage_kernels(idx_sim* s, int mode) {
  if (!s || mode < 0 || mode > 3) return IDX_EINVAL;
  if (mode == 2 && !s->fused_ok) return IDX_EINVAL;
  if (mode == 3 && !s->carry_ok) return IDX_EINVAL;
  s->stage_mode = mode;
  choose_stage_kernels(s);
  // the captured cycle holds the old kernels
  if (s->exec) { cudaGraphExecDestroy(s->exec); s->exec = nullptr; }
  if (s->graph) { cudaGraphDestroy(s->graph); s->graph = nullptr; }
  return IDX_OK;
}

int idx_stage_kernels(const idx_sim* cs, int* in_use) {
  idx_sim* s = const_cast<idx_sim*>(cs);
  if (!s || !in_use) return IDX_EINVAL;
  choose_stage_kernels(s);
  *in_use = s->use_fused ? 2 : (s->use_carry ? 3 : 1);
  return IDX_OK;
}

int idx_step_count(const idx_sim* cs, int64_t* nsteps) {
  idx_sim* s = const_cast<idx_sim*>(cs);
  if (!s || !nsteps) return IDX_EINVAL;
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  *nsteps = (int64_t)s->host_ctrl->nsteps;
  return pending_error(s);
}

int idx_footprint(const idx_grid* grid, int precision, uint64_t* bytes) {
  if (!grid || !bytes || grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return IDX_EINVAL;
  if (precision != IDX_FP64 && precision != IDX_FP32_BULK) return IDX_EINVAL;
  int bc[3], pn[3];
  if (!grid_bc(grid, bc, pn)) return IDX_EINVAL;
  const long long ncell = (long long)pn[0] * pn[1] * pn[2];
  if (ncell >= (1ll << 31)) return IDX_EINVAL;
  const bool bounded = bc[0] || bc[1] || bc[2];
  *bytes = (uint64_t)sim_bytes(ncell, precision == IDX_FP32_BULK, false, false, bounded);
  return IDX_OK;
}

int idx_footprint_solver(const idx_grid* grid, const idx_solver* solver, uint64_t* bytes) {
  if (!grid || !bytes || !valid_solver(solver) || grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
    return IDX_EINVAL;
  int bc[3], pn[3];
  if (!grid_bc(grid, bc, pn)) return IDX_EINVAL;
  const long long ncell = (long long)pn[0] * pn[1] * pn[2];
  if (ncell >= (1ll << 31)) return IDX_EINVAL;
  const bool bounded = bc[0] || bc[1] || bc[2];
  *bytes = (uint64_t)sim_bytes(ncell, solver->precision == IDX_FP32_BULK, solver->rk_order == 3,
                               solver->induction == IDX_INDUCTION_POTENTIAL, bounded);
  return IDX_OK;
}

int idx_last_error_cell(const idx_sim* s, int64_t* cell) {
  if (!s || !cell) return IDX_EINVAL;
  *cell = s->last_bad;
  return IDX_OK;
}

int idx_get_clock(const idx_sim* cs, idx_clock* clock) {
  idx_sim* s = const_cast<idx_sim*>(cs);
  if (!s || !clock) return IDX_EINVAL;
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  rc = pending_error(s);
  if (rc != IDX_OK) return rc;
  clock->t = s->host_ctrl->t;
  std::memcpy(&clock->inv_dt, &s->host_ctrl->inv_prev, sizeof(double));
  clock->nsteps = (int64_t)s->host_ctrl->nsteps;
  return IDX_OK;
}

int idx_set_clock(idx_sim* s, const idx_clock* clock) {
  if (!s || !clock || !std::isfinite(clock->t) || !(clock->inv_dt > 0.0) ||
      !std::isfinite(clock->inv_dt) || clock->nsteps < 0)
    return IDX_EINVAL;
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  rc = pending_error(s);
  if (rc != IDX_OK) return rc;
  Ctrl c = *s->host_ctrl;
  c.t = clock->t;
  std::memcpy(&c.inv_prev, &clock->inv_dt, sizeof(double));
  c.nsteps = (long long)clock->nsteps;
  c.done = 0;
  IDX_TRY(cudaMemcpyAsync(s->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream));
  return sync_ctrl(s);
}

}  // extern "C"

// ===========================================================================
// idx_probe_bounded_wait: the bounded mbarrier wait of the staged sweeps, run alone in
// one block, so that tests can make it expire without a fault.  The block initialises
// an mbarrier, announces `announce` transaction bytes and issues no copy: with bytes
// announced the phase cannot complete, the wait gives up after limit_ns, and the block
// records IDX_ETIMEOUT in its control block through the same give-up path as the
// sweeps (which waits once more, bounded, for copies in flight -- there are none).
// With announce == 0 the phase completes at once and nothing is recorded.
// ===========================================================================
namespace {
__global__ void k_wait_probe(Ctrl* ctrl, uint32_t announce, uint64_t limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, announce);
  const bool landed = mbar_wait(&bar, 0, limit_ns);
  if (__syncthreads_or(!landed)) {
    if (threadIdx.x == 0) flag_timeout(ctrl);
    mbar_wait(&bar, 0, limit_ns);  // copies in flight: none were issued
  }
}
}  // namespace

extern "C" int idx_probe_bounded_wait(void* stream, uint32_t announce_bytes, double limit_ms) {
  if (!(limit_ms > 0.0) || !(limit_ms <= 1000.0) || announce_bytes >= (1u << 20)) return IDX_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  Ctrl* d = nullptr;
  if (cudaMallocAsync(&d, sizeof(Ctrl), st) != cudaSuccess) {
    cudaGetLastError();
    return IDX_ENOMEM;
  }
  Ctrl h;
  std::memset(&h, 0, sizeof(h));
  int rc = IDX_OK;
  if (cudaMemcpyAsync(d, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = IDX_ECUDA;
  if (rc == IDX_OK) {
    k_wait_probe<<<1, 64, 0, st>>>(d, announce_bytes, (uint64_t)(limit_ms * 1e6));
    if (cudaGetLastError() != cudaSuccess) rc = IDX_ECUDA;
  }
  if (rc == IDX_OK && cudaMemcpyAsync(&h, d, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    rc = IDX_ECUDA;
  cudaFreeAsync(d, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) rc = IDX_ECUDA;
  if (rc != IDX_OK) return rc;
  return h.err;
}

// ===========================================================================
// idx_step_noalloc: one FP64 cycle on caller-owned device state with no allocation.
// For callers that cannot allocate device memory (another framework's pool, a device
// budget, or a latency-bound path).  The scratch of the cycle lives in a file-scope
// device array held by every GPU that loads the library; see include/idx.h.
// ===========================================================================
namespace {

constexpr size_t kNoAllocBytes = IDX_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoAllocArrays = 8 + 8 + 24 + 3;  // U1, W, F (3 x 8), E (3)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
static_assert(256 + kNoAllocArrays * align256(sizeof(double) * (size_t)IDX_NOALLOC_MAX_CELLS) <=
                  kNoAllocBytes,
              "IDX_NOALLOC_MAX_CELLS does not fit the scratch array");
static_assert(sizeof(Ctrl) <= 256, "control block must fit its 256-byte slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// In host code g_noalloc_scratch names a host-side stand-in, not device memory: the
// device address is looked up once per device and CUDA context (with that device
// current) and cached.  Each context that loads the library's module has its own copy of
// the array at its own address, so a caller that makes another context current (another
// framework's own context) gets that context's copy.
using CtxGetCurrent = CUresult (*)(CUcontext*);

CtxGetCurrent ctx_get_current() {
  static CtxGetCurrent fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrent>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

std::map<std::pair<int, CUcontext>, void*> g_noalloc_addr;
std::mutex g_noalloc_mutex;

int noalloc_scratch(int device, void** out) {
  CtxGetCurrent get = ctx_get_current();
  CUcontext ctx = nullptr;
  // the runtime makes the device's primary context current on first use
  if (cudaFree(nullptr) != cudaSuccess) return IDX_ECUDA;
  if (!get || get(&ctx) != CUDA_SUCCESS) return IDX_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  const auto key = std::make_pair(device, ctx);
  auto it = g_noalloc_addr.find(key);
  if (it == g_noalloc_addr.end()) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return IDX_ECUDA;
    it = g_noalloc_addr.emplace(key, p).first;
  }
  *out = it->second;
  return IDX_OK;
}

}  // namespace

extern "C" int idx_step_noalloc(const idx_grid* grid, double gamma, double cfl,
                                double* const state[8], double* inv_dt, double* dt_taken,
                                void* stream) {
  if (!grid || !state || !inv_dt || !(gamma > 1.0) || !std::isfinite(gamma) ||
      !(cfl > 0.0 && cfl < 1.0))
    return IDX_EINVAL;
  for (int f = 0; f < 8; ++f)
    if (!state[f]) return IDX_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return IDX_EINVAL;
  if (!(grid->lx > 0) || !(grid->ly > 0) || !(grid->lz > 0)) return IDX_EINVAL;
  {
    int bc[3], pn[3];
    if (!grid_bc(grid, bc, pn) || bc[0] || bc[1] || bc[2]) return IDX_EINVAL;
  }
  const long long ncell = (long long)grid->nx * grid->ny * grid->nz;
  if (ncell > IDX_NOALLOC_MAX_CELLS) return IDX_ETOOLARGE;
  {
    // the call reads back the control block and waits for its stream: neither may be
    // recorded into a graph, so a stream that is capturing is refused
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) return IDX_ECUDA;
    if (cap != cudaStreamCaptureStatusNone) return IDX_EINVAL;
  }

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return IDX_ECUDA;
  void* base = nullptr;
  int rc = noalloc_scratch(device, &base);
  if (rc != IDX_OK) return rc;

  // a sim descriptor on the host stack whose buffers point into the scratch array
  idx_sim s;
  std::memset(&s, 0, sizeof(s));
  s.grid = *grid;
  s.gamma = gamma;
  s.solver.recon = 1; s.solver.riemann = 4; s.solver.emf = 2; s.solver.rk_order = 2;
  s.solver.cfl = cfl; s.solver.precision = IDX_FP64;
  s.stream = (cudaStream_t)stream;
  s.device = device;
  Geo& g = s.geo;
  g.n[0] = grid->nx; g.n[1] = grid->ny; g.n[2] = grid->nz;
  g.stride[0] = 1; g.stride[1] = grid->nx; g.stride[2] = grid->nx * grid->ny;
  g.ncell = (int)ncell;
  geo_set_divisors(g);
  const double l[3] = {grid->lx, grid->ly, grid->lz};
  for (int d = 0; d < 3; ++d) {
    g.active[d] = g.n[d] > 1;
    g.inv_dl[d] = (double)g.n[d] / l[d];
    g.dl[d] = l[d] / (double)g.n[d];
    g.inv_dlf[d] = (float)g.inv_dl[d];
  }
  geo_set_gamma(g, gamma);
  g.riemann = 4;
  g.recon = 1;
  const size_t arr = align256(sizeof(double) * (size_t)ncell);
  char* p = (char*)base;
  s.ctrl = (Ctrl*)p;
  p += 256;
  for (int f = 0; f < 8; ++f) s.U.f[f] = state[f];
  for (int f = 0; f < 8; ++f) { s.U1.f[f] = (double*)p; p += arr; }
  for (int f = 0; f < 8; ++f) { s.Wd.f[f] = (double*)p; p += arr; }
  for (int d = 0; d < 3; ++d)
    for (int f = 0; f < 8; ++f) { s.Fd[d].f[f] = (double*)p; p += arr; }
  for (int d = 0; d < 3; ++d) { s.Ed[d] = (double*)p; p += arr; }

  // The array keeps the previous call's contents.  Only the control block must start
  // from a known value; every other array is written before it is read in the cycle.
  Ctrl c;
  std::memset(&c, 0, sizeof(c));
  c.t_end = std::numeric_limits<double>::infinity();
  c.cfl = cfl;
  c.bad_cell = ~0ull;
  c.bad_next = ~0ull;
  if (*inv_dt > 0.0) std::memcpy(&c.inv_prev, inv_dt, sizeof(double));
  IDX_TRY(cudaMemcpyAsync(s.ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, s.stream));
  if (!(*inv_dt > 0.0)) {
    // no bound carried in: the signal-speed pass of a first cycle
    launch_speed_pass<double>(&s, s.U, s.Wd, s.Fd);
  }
  launch_cycle(&s);
  IDX_TRY(cudaGetLastError());
  Ctrl out;
  IDX_TRY(cudaMemcpyAsync(&out, s.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s.stream));
  IDX_TRY(cudaStreamSynchronize(s.stream));
  if (out.err != 0) return out.err;
  std::memcpy(inv_dt, &out.inv_prev, sizeof(double));
  if (dt_taken) *dt_taken = out.last_dt;
  return IDX_OK;
}

// ===========================================================================
// Batched stepping (idx_batch_*): many sims -- each with its own grid, state,
// scratch, control block, dt and end time -- advanced together.  Per stage every
// kernel type is launched once, as a grid-stride loop of resident blocks over a
// device work-list of (instance, first index) items of kThreads cells or sweep
// threads.  The work-list is read at run time, so one captured graph of a batched
// cycle serves every membership: instances join and leave between graph replays by
// rewriting the list, without re-capture.  The per-cell arithmetic is the same device
// code as the single-sim kernels, so a sim gives the same result, to rounding (FMA
// contraction may differ between kernel instantiations), alone and in a batch.  The FP32
// work-list kernels carry a member's header in registers beside the cell's arithmetic;
// their launch bounds hold them to 3-6 resident blocks per SM (a few spilled words), which
// measured faster on the batched mix than the 2-3 blocks their register counts gave.
// ===========================================================================
namespace {

template <typename T> struct InstT {
  CUtensorMap tm_body[3][2];  // the member's staged-sweep maps (global memory copies)
  CUtensorMap tm_halo[3];
  Geo g;
  Ptr8<double> U, U1;
  Ptr8<T> W;
  Ptr8<T> F[3];
  T* E[3];
  CellEmf<T> cc;
  Ctrl* ctrl;
};

struct Item {
  int inst;
  int begin;
};

template <typename T> struct BatchDev {
  InstT<T>* inst;
  Item* cell;      // items of kThreads cells
  Item* sweep[3];  // items of kThreads marching/warp sweep threads, per direction
  Item* tile[3];   // items of one staged tile (begin = tile index), per direction
  Ctrl* gather;    // poll buffer, one Ctrl per instance
  int n_inst;
  int n_cell;
  int n_sweep[3];
  int n_tile[3];
};

template <typename T> __device__ __forceinline__ Ptr8<const T> dconst(const Ptr8<T>& p) {
  Ptr8<const T> q;
#pragma unroll
  for (int f = 0; f < 8; ++f) q.f[f] = p.f[f];
  return q;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 6 : 1) kb_prims(const BatchDev<T>* B, int stage, int check) {
  const int n = B->n_cell;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const Item w = B->cell[it];
    const InstT<T>* I = &B->inst[w.inst];
    if (check && !(I->ctrl->dt > 0.0)) continue;
    const Geo g = I->g;
    const int c = w.begin + threadIdx.x;
    if (c < g.ncell) prims_body<T>(g, dconst(stage ? I->U1 : I->U), I->W, I->cc, I->ctrl, c);
  }
}

template <typename T, int D, int SEG>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 1) kb_sweep(const BatchDev<T>* B, int stage, int check) {
  const int n = B->n_sweep[D];
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const Item w = B->sweep[D][it];
    const InstT<T>* I = &B->inst[w.inst];
    if (check && !(I->ctrl->dt > 0.0)) continue;
    const Geo g = I->g;
    const double* bface = (stage ? I->U1 : I->U).f[5 + D];
    if (SEG > 0)
      sweep_body<T, D, (SEG > 0 ? SEG : 1)>(g, dconst(I->W), bface, I->F[D], w.begin + threadIdx.x);
    else
      sweep_x_body<T>(g, dconst(I->W), bface, I->F[D], w.begin + threadIdx.x);
  }
}

// Staged sweep over the batch's tile items (members whose grids fit the tiles): a
// persistent block refills its shared-memory tile item after item, the mbarrier's phase
// parity flipping with each completed copy.
template <typename T, int D, int L>
__global__ void __launch_bounds__(8 * L, sizeof(T) == 4 ? 96 / L : 1)
    kb_sweep_tma(const BatchDev<T>* B, int stage, int check) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  const int n = B->n_tile[D];
  uint32_t parity = 0;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const Item w = B->tile[D][it];
    const InstT<T>* I = &B->inst[w.inst];
    if (check && !(I->ctrl->dt > 0.0)) continue;  // uniform over the block
    const Geo g = I->g;
    const double* bface = (stage ? I->U1 : I->U).f[5 + D];
    if (!tma_tile<T, D, L>(g, &I->tm_body[D][L == 32 ? 1 : 0], &I->tm_halo[D], bface, I->F[D],
                           w.begin, tile, &bar, parity)) {
      tma_give_up(I->ctrl, &bar, parity);
      return;
    }
    parity ^= 1u;
    __syncthreads();  // every thread is done with the tile before it is refilled
    if (threadIdx.x == 0) fence_proxy_async();
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 5 : 1) kb_emf(const BatchDev<T>* B) {
  const int n = B->n_cell;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const Item w = B->cell[it];
    const InstT<T>* I = &B->inst[w.inst];
    if (!(I->ctrl->dt > 0.0)) continue;
    const Geo g = I->g;
    const int c = w.begin + threadIdx.x;
    if (c < g.ncell)
      emf_body<T>(g, dconst(I->W), dconst(I->F[0]), dconst(I->F[1]), dconst(I->F[2]), I->cc, I->E[0],
                  I->E[1], I->E[2], c);
  }
}

template <typename T, bool COMBINE>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 1) kb_update(const BatchDev<T>* B) {
  const int n = B->n_cell;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const Item w = B->cell[it];
    const InstT<T>* I = &B->inst[w.inst];
    const double dt = I->ctrl->dt;
    if (!(dt > 0.0)) continue;  // uniform over the block: one item per block
    const Geo g = I->g;
    const T inv = update_body<T, COMBINE, false, false>(
        g, dconst(COMBINE ? I->U1 : I->U), dconst(I->U), dconst(I->F[0]), dconst(I->F[1]),
        dconst(I->F[2]), I->E[0], I->E[1], I->E[2], COMBINE ? I->U : I->U1, dt,
        w.begin + threadIdx.x);
    block_max_to(&I->ctrl->inv_acc, inv);
  }
}

template <typename T> __global__ void kb_begin(const BatchDev<T>* B) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B->n_inst; i += gridDim.x * blockDim.x)
    begin_body(B->inst[i].ctrl);
}

template <typename T> __global__ void kb_end(const BatchDev<T>* B) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B->n_inst; i += gridDim.x * blockDim.x)
    end_body(B->inst[i].ctrl);
}

template <typename T> __global__ void kb_gather(const BatchDev<T>* B) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B->n_inst; i += gridDim.x * blockDim.x)
    B->gather[i] = *B->inst[i].ctrl;
}

}  // namespace

constexpr int kSoloStreams = 4;

struct idx_batch {
  int precision;
  cudaStream_t stream;
  bool own_stream;
  // the solo members' stages, forked from and joined to stream over kSoloStreams streams
  cudaStream_t side[kSoloStreams] = {};
  cudaEvent_t fork_ev = nullptr, join_ev[kSoloStreams] = {};
  int device;
  int sms;
  std::vector<idx_sim*> sims;
  void* header;        // BatchDev<T>, fixed address (captured by the graph)
  void* lists;         // instances, items, poll buffer (reallocated as the batch grows)
  size_t lists_cap;
  Ctrl* host_gather;   // pinned
  size_t host_cap;
  bool dirty;
  bool tuned;
  int shape[3];        // sweep shape per direction (marching segment, -1 warp x sweep,
                       // 116 / 132 staged tiles for the members that fit them)
  int fallback[3];     // marching shape of the other members when shape[d] is staged
  int graph_shape[3], graph_fallback[3];
  int grid_tma[2];     // persistent blocks of the staged sweep, L = 16 / 32
  std::vector<idx_sim*> solo;        // members stepped by their own kernels in the cycle
  std::vector<uint64_t> graph_solo;  // serials of the solo members the captured cycle holds
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int grid_cell, grid_sweep;
};

namespace {

template <typename T> InstT<T> inst_of(idx_sim* s);

std::vector<std::vector<idx_sim*>> solo_lanes(const idx_batch* b) {
  std::vector<idx_sim*> order(b->solo.begin(), b->solo.end());
  std::stable_sort(order.begin(), order.end(), [](const idx_sim* a, const idx_sim* c) {
    return a->geo.ncell > c->geo.ncell;
  });
  std::vector<std::vector<idx_sim*>> lanes(kSoloStreams);
  std::vector<long long> load(kSoloStreams, 0);
  for (idx_sim* s : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[k].push_back(s);
    load[k] += s->geo.ncell;
  }
  return lanes;
}

// Members of at least this many cells run the single-sim kernels inside the batched cycle:
// their own launch parameters and tuned shapes beat the work-list kernels once a member
// fills the GPU by itself (measured on the FP32-bulk boxes of 32^3 .. 128^3), while the
// small members gain most from sharing launches.
constexpr int kSoloCells = 1 << 18;
template <typename T> void copy_maps(InstT<T>& I, const idx_sim* s) {
  for (int d = 0; d < 3; ++d) {
    I.tm_body[d][0] = s->tm_body[d][0];
    I.tm_body[d][1] = s->tm_body[d][1];
    I.tm_halo[d] = s->tm_halo[d];
  }
}
template <> InstT<double> inst_of<double>(idx_sim* s) {
  InstT<double> I;
  copy_maps(I, s);
  I.g = s->geo; I.U = s->U; I.U1 = s->U1; I.W = s->Wd;
  for (int d = 0; d < 3; ++d) { I.F[d] = s->Fd[d]; I.E[d] = s->Ed[d]; }
  I.cc = s->Cd;
  I.ctrl = s->ctrl;
  return I;
}
template <> InstT<float> inst_of<float>(idx_sim* s) {
  InstT<float> I;
  copy_maps(I, s);
  I.g = s->geo; I.U = s->U; I.U1 = s->U1; I.W = s->Wf;
  for (int d = 0; d < 3; ++d) { I.F[d] = s->Ff[d]; I.E[d] = s->Ef[d]; }
  I.cc = s->Cf;
  I.ctrl = s->ctrl;
  return I;
}

int sweep_threads(const Geo& g, int d, int shape) {
  if (shape == -1 && d == 0) return warpx_threads(g);
  return march_threads(g, d, shape > 0 ? shape : kSegDefault);
}

// Build the work-lists on the host and upload them with the header.
template <typename T> int batch_upload(idx_batch* b) {
  const int n = (int)b->sims.size();
  std::vector<InstT<T>> inst(n);
  std::vector<Item> cell, sweep[3], tile[3];
  b->solo.clear();
  for (int i = 0; i < n; ++i) {
    idx_sim* s = b->sims[i];
    inst[i] = inst_of<T>(s);
    // stepped by its own kernels, no work-list items: large members, and members whose
    // cycle the work-list kernels do not run (RK3, vector-potential form, LimO3, boundaries)
    if (s->geo.ncell >= kSoloCells || s->solver.rk_order != 2 || s->pot || s->bounded ||
        s->geo.recon != 1) {
      b->solo.push_back(s);
      continue;
    }
    for (int c0 = 0; c0 < s->geo.ncell; c0 += kThreads) cell.push_back({i, c0});
    for (int d = 0; d < 3; ++d) {
      if (!s->geo.active[d]) continue;
      const int sd = b->shape[d];
      const bool staged = d != 0 && (sd == 116 || sd == 132);
      if (staged && tma_shape_ok(s, d, sd)) {
        const Geo& g = s->geo;
        const int ntiles = (g.n[0] / 32) * (g.n[d] / (sd - 100)) * g.n[d == 1 ? 2 : 1];
        for (int t = 0; t < ntiles; ++t) tile[d].push_back({i, t});
        continue;
      }
      const int nt = sweep_threads(s->geo, d, staged ? b->fallback[d] : sd);
      for (int t0 = 0; t0 < nt; t0 += kThreads) sweep[d].push_back({i, t0});
    }
  }
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t need = al(sizeof(InstT<T>) * (n + 1)) + al(sizeof(Item) * (cell.size() + 1)) +
                al(sizeof(Ctrl) * (n + 1));
  for (int d = 0; d < 3; ++d)
    need += al(sizeof(Item) * (sweep[d].size() + 1)) + al(sizeof(Item) * (tile[d].size() + 1));
  if (need > b->lists_cap) {
    IDX_TRY(cudaStreamSynchronize(b->stream));
    if (b->lists) cudaFree(b->lists);
    b->lists = nullptr;
    b->lists_cap = 0;
    if (cudaMalloc(&b->lists, 2 * need) != cudaSuccess) {
      cudaGetLastError();
      return IDX_ENOMEM;
    }
    b->lists_cap = 2 * need;
  }
  if ((size_t)n * sizeof(Ctrl) > b->host_cap) {
    IDX_TRY(cudaStreamSynchronize(b->stream));
    if (b->host_gather) cudaFreeHost(b->host_gather);
    b->host_gather = nullptr;
    b->host_cap = 0;
    if (cudaMallocHost(&b->host_gather, 2 * (n + 1) * sizeof(Ctrl)) != cudaSuccess) return IDX_ENOMEM;
    b->host_cap = 2 * (n + 1) * sizeof(Ctrl);
  }
  BatchDev<T> h;
  char* p = (char*)b->lists;
  h.inst = (InstT<T>*)p; p += al(sizeof(InstT<T>) * (n + 1));
  h.cell = (Item*)p; p += al(sizeof(Item) * (cell.size() + 1));
  for (int d = 0; d < 3; ++d) { h.sweep[d] = (Item*)p; p += al(sizeof(Item) * (sweep[d].size() + 1)); }
  for (int d = 0; d < 3; ++d) { h.tile[d] = (Item*)p; p += al(sizeof(Item) * (tile[d].size() + 1)); }
  h.gather = (Ctrl*)p;
  h.n_inst = n;
  h.n_cell = (int)cell.size();
  for (int d = 0; d < 3; ++d) h.n_sweep[d] = (int)sweep[d].size();
  for (int d = 0; d < 3; ++d) h.n_tile[d] = (int)tile[d].size();
  // pageable sources: each copy is staged before the call returns
  if (n) IDX_TRY(cudaMemcpyAsync(h.inst, inst.data(), sizeof(InstT<T>) * n, cudaMemcpyHostToDevice, b->stream));
  if (!cell.empty()) IDX_TRY(cudaMemcpyAsync(h.cell, cell.data(), sizeof(Item) * cell.size(), cudaMemcpyHostToDevice, b->stream));
  for (int d = 0; d < 3; ++d) {
    if (!sweep[d].empty())
      IDX_TRY(cudaMemcpyAsync(h.sweep[d], sweep[d].data(), sizeof(Item) * sweep[d].size(), cudaMemcpyHostToDevice, b->stream));
    if (!tile[d].empty())
      IDX_TRY(cudaMemcpyAsync(h.tile[d], tile[d].data(), sizeof(Item) * tile[d].size(), cudaMemcpyHostToDevice, b->stream));
  }
  IDX_TRY(cudaMemcpyAsync(b->header, &h, sizeof(h), cudaMemcpyHostToDevice, b->stream));
  IDX_TRY(cudaStreamSynchronize(b->stream));
  return IDX_OK;
}

template <typename T, int D>
void launch_batch_sweep_d(idx_batch* b, int shape, int stage, int check) {
  const BatchDev<T>* B = (const BatchDev<T>*)b->header;
  const int grid = b->grid_sweep;
  switch (shape) {
    case -1: if (D == 0) { kb_sweep<T, D, -1><<<grid, kThreads, 0, b->stream>>>(B, stage, check); return; } break;
    case 2: kb_sweep<T, D, 2><<<grid, kThreads, 0, b->stream>>>(B, stage, check); return;
    case 4: kb_sweep<T, D, 4><<<grid, kThreads, 0, b->stream>>>(B, stage, check); return;
    case 8: kb_sweep<T, D, 8><<<grid, kThreads, 0, b->stream>>>(B, stage, check); return;
    case 32: kb_sweep<T, D, 32><<<grid, kThreads, 0, b->stream>>>(B, stage, check); return;
    default: break;
  }
  kb_sweep<T, D, kSegDefault><<<grid, kThreads, 0, b->stream>>>(B, stage, check);
}

template <typename T, int D, int L> void launch_batch_tma(idx_batch* b, int stage, int check) {
  const BatchDev<T>* B = (const BatchDev<T>*)b->header;
  const size_t smem = 7 * (L + 4) * 32 * sizeof(T);
  kb_sweep_tma<T, D, L><<<b->grid_tma[L == 32 ? 1 : 0], 8 * L, smem, b->stream>>>(B, stage, check);
}

// A staged shape launches the tile kernel for the members that fit the tiles and the
// marching fallback for the others (each loops over an empty list when it has none).
template <typename T> void launch_batch_sweep(idx_batch* b, int d, int stage, int check) {
  const int sd = b->shape[d];
  if (d != 0 && (sd == 116 || sd == 132)) {
    if (d == 1) {
      if (sd == 116) launch_batch_tma<T, 1, 16>(b, stage, check);
      else launch_batch_tma<T, 1, 32>(b, stage, check);
      launch_batch_sweep_d<T, 1>(b, b->fallback[1], stage, check);
    } else {
      if (sd == 116) launch_batch_tma<T, 2, 16>(b, stage, check);
      else launch_batch_tma<T, 2, 32>(b, stage, check);
      launch_batch_sweep_d<T, 2>(b, b->fallback[2], stage, check);
    }
    return;
  }
  if (d == 0) launch_batch_sweep_d<T, 0>(b, sd, stage, check);
  else if (d == 1) launch_batch_sweep_d<T, 1>(b, sd, stage, check);
  else launch_batch_sweep_d<T, 2>(b, sd, stage, check);
}

// The stages of one solo member's own cycle (its RK order and induction form), on stream
// st (and into the batch's graph).
void launch_solo_stages(idx_sim* s, cudaStream_t st) {
  const cudaStream_t own = s->stream;
  s->stream = st;
  if (s->use_carry) {
    launch_carry_stages(s);
    s->stream = own;
    return;
  }
  const StagePlan p = stage_plan(s);
  for (int q = 0; q < p.n; ++q) {
    if (s->solver.precision == IDX_FP32_BULK) launch_stage<float>(s, p, q, s->Wf, s->Ff, s->Ef);
    else launch_stage<double>(s, p, q, s->Wd, s->Fd, s->Ed);
  }
  s->stream = own;
}

// Solo members over the side streams: largest first, each onto the stream with the fewest
// cells so far, so that members' kernels run side by side and fill each other's tails.
std::vector<std::vector<idx_sim*>> solo_lanes(const idx_batch* b);

// One batched cycle: every member's dt, then -- side by side -- both RK2 stages of the
// work-list members on the batch stream and each solo member's own stages on the side
// streams (they touch disjoint buffers and need only the dt), then every member's time and
// speeds.  The solo kernels fill the SMs that the work-list kernels and each other leave
// idle in their tails; in the captured graph the forks and joins are edges.
template <typename T> void launch_batch_cycle(idx_batch* b) {
  const BatchDev<T>* B = (const BatchDev<T>*)b->header;
  kb_begin<T><<<b->sms, kThreads, 0, b->stream>>>(B);
  const bool fork = !b->solo.empty() && b->side[0];
  int used = 0;
  if (fork) {
    cudaEventRecord(b->fork_ev, b->stream);
    const std::vector<std::vector<idx_sim*>> lanes = solo_lanes(b);
    for (size_t k = 0; k < lanes.size(); ++k) {
      if (lanes[k].empty()) continue;
      cudaStreamWaitEvent(b->side[k], b->fork_ev, 0);
      for (idx_sim* s : lanes[k]) launch_solo_stages(s, b->side[k]);
      cudaEventRecord(b->join_ev[k], b->side[k]);
      used |= 1 << k;
    }
  }
  for (int st = 0; st < 2; ++st) {
    kb_prims<T><<<b->grid_cell, kThreads, 0, b->stream>>>(B, st, 1);
    for (int d = 0; d < 3; ++d) launch_batch_sweep<T>(b, d, st, 1);
    kb_emf<T><<<b->grid_cell, kThreads, 0, b->stream>>>(B);
    if (st == 0) kb_update<T, false><<<b->grid_cell, kThreads, 0, b->stream>>>(B);
    else kb_update<T, true><<<b->grid_cell, kThreads, 0, b->stream>>>(B);
  }
  if (fork) {
    for (int k = 0; k < kSoloStreams; ++k)
      if (used & (1 << k)) cudaStreamWaitEvent(b->stream, b->join_ev[k], 0);
  } else {
    for (idx_sim* s : b->solo) launch_solo_stages(s, b->stream);
  }
  kb_end<T><<<b->sms, kThreads, 0, b->stream>>>(B);
}

// Tile-shape autotuner of the batch: per direction, every candidate sweep shape is timed
// on the whole batch (primitives of the current states, three launches each).
template <typename T> int batch_tune(idx_batch* b) {
  const BatchDev<T>* B = (const BatchDev<T>*)b->header;
  int rc = batch_upload<T>(b);
  if (rc != IDX_OK) return rc;
  kb_prims<T><<<b->grid_cell, kThreads, 0, b->stream>>>(B, 0, 0);
  cudaEvent_t e0, e1;
  IDX_TRY(cudaEventCreate(&e0));
  IDX_TRY(cudaEventCreate(&e1));
  const int cand[6] = {-1, 2, 4, 8, 16, 32};
  for (int d = 0; d < 3 && rc == IDX_OK; ++d) {
    bool any = false;
    for (idx_sim* s : b->sims) any = any || s->geo.active[d];
    if (!any) continue;
    float best = 1e30f;
    int best_shape = kSegDefault;
    for (int q = 0; q < 6 && rc == IDX_OK; ++q) {
      if (cand[q] == -1 && d != 0) continue;
      b->shape[d] = cand[q];
      rc = batch_upload<T>(b);
      if (rc != IDX_OK) break;
      launch_batch_sweep<T>(b, d, 0, 0);
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 3; ++r) launch_batch_sweep<T>(b, d, 0, 0);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = IDX_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_shape = cand[q]; }
    }
    b->shape[d] = best_shape;
    // staged tiles for the members that fit them, the best marching shape for the rest
    if (d == 0 || rc != IDX_OK) continue;
    const int march = best_shape;
    for (const int staged : {116, 132}) {
      bool fits = false;
      for (idx_sim* s : b->sims) fits = fits || (s->geo.active[d] && tma_shape_ok(s, d, staged));
      if (!fits) continue;
      b->shape[d] = staged;
      b->fallback[d] = march;
      rc = batch_upload<T>(b);
      if (rc != IDX_OK) break;
      launch_batch_sweep<T>(b, d, 0, 0);
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < 3; ++r) launch_batch_sweep<T>(b, d, 0, 0);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { rc = IDX_ECUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_shape = staged; }
    }
    b->shape[d] = best_shape;
    b->fallback[d] = march;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != IDX_OK) return rc;
  IDX_TRY(cudaGetLastError());
  b->tuned = true;
  return batch_upload<T>(b);
}

template <typename T> int batch_prepare(idx_batch* b) {
  if (b->dirty) {
    int rc = (!b->tuned && !b->sims.empty()) ? batch_tune<T>(b) : batch_upload<T>(b);
    if (rc != IDX_OK) return rc;
    b->dirty = false;
  }
  // solo members' own shapes, tuned before the capture (cached per grid); the primitives
  // of a carried-primitive member's state before its first batched cycle
  for (idx_sim* s : b->solo) {
    const int trc = tune_once(s);
    if (trc != IDX_OK) return trc;
    refresh_carry(s, b->stream);
  }
  std::vector<uint64_t> solo_serials;
  for (const idx_sim* s : b->solo) solo_serials.push_back(s->serial);
  bool same = b->exec != nullptr && b->graph_solo == solo_serials;
  for (int d = 0; d < 3; ++d)
    same = same && b->graph_shape[d] == b->shape[d] && b->graph_fallback[d] == b->fallback[d];
  if (same) return IDX_OK;
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  IDX_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  launch_batch_cycle<T>(b);
  IDX_TRY(cudaStreamEndCapture(b->stream, &b->graph));
  IDX_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  for (int d = 0; d < 3; ++d) {
    b->graph_shape[d] = b->shape[d];
    b->graph_fallback[d] = b->fallback[d];
  }
  b->graph_solo = solo_serials;
  return IDX_OK;
}

// The FP64 tiles of 32 rows take 63 KB of shared memory, above the 48 KB default.
void allow_batch_tma_smem() {
  const int big = 7 * (32 + 4) * 32 * (int)sizeof(double);
  cudaFuncSetAttribute(kb_sweep_tma<double, 1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(kb_sweep_tma<double, 2, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaGetLastError();
}

template <typename T> int batch_occupancy(idx_batch* b) {
  allow_batch_tma_smem();
  int per_sm_cell = 0, per_sm_sweep = 0;
  IDX_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_cell, kb_update<T, true>, kThreads, 0));
  IDX_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_sweep, kb_sweep<T, 1, kSegDefault>, kThreads, 0));
  b->grid_cell = b->sms * (per_sm_cell > 0 ? per_sm_cell : 1);
  b->grid_sweep = b->sms * (per_sm_sweep > 0 ? per_sm_sweep : 1);
  int per16 = 0, per32 = 0;
  IDX_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per16, kb_sweep_tma<T, 1, 16>, 8 * 16,
                                                        7 * 20 * 32 * sizeof(T)));
  IDX_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per32, kb_sweep_tma<T, 1, 32>, 8 * 32,
                                                        7 * 36 * 32 * sizeof(T)));
  b->grid_tma[0] = b->sms * (per16 > 0 ? per16 : 1);
  b->grid_tma[1] = b->sms * (per32 > 0 ? per32 : 1);
  return IDX_OK;
}

// Set a member's end time (and clear its done flag when it still has time to go).
int arm_end_time(cudaStream_t stream, idx_sim* s, double t_end) {
  int rc = sync_ctrl(s);
  if (rc != IDX_OK) return rc;
  Ctrl c = *s->host_ctrl;
  c.t_end = t_end;
  c.done = (c.t >= t_end) ? 1 : 0;
  IDX_TRY(cudaMemcpyAsync(s->ctrl, &c, sizeof(Ctrl), cudaMemcpyHostToDevice, stream));
  IDX_TRY(cudaStreamSynchronize(stream));
  return IDX_OK;
}

}  // namespace

extern "C" {

int idx_batch_create(int precision, void* stream, idx_batch** out) {
  if (!out || (precision != IDX_FP64 && precision != IDX_FP32_BULK)) return IDX_EINVAL;
  *out = nullptr;
  idx_batch* b = new idx_batch();
  b->precision = precision;
  b->dirty = true;
  for (int d = 0; d < 3; ++d) {
    b->shape[d] = b->fallback[d] = kSegDefault;
    b->graph_shape[d] = b->graph_fallback[d] = 0;
  }
  int rc = IDX_OK;
  if (cudaGetDevice(&b->device) != cudaSuccess) rc = IDX_ECUDA;
  if (rc == IDX_OK && cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) rc = IDX_ECUDA;
  if (rc == IDX_OK) {
    if (stream) {
      b->stream = (cudaStream_t)stream;
    } else {
      b->own_stream = true;
      if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) rc = IDX_ECUDA;
    }
  }
  if (rc == IDX_OK && cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess)
    rc = IDX_ECUDA;
  for (int k = 0; k < kSoloStreams && rc == IDX_OK; ++k)
    if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
      rc = IDX_ECUDA;
  if (rc == IDX_OK && cudaMalloc(&b->header, 256) != cudaSuccess) rc = IDX_ENOMEM;
  if (rc == IDX_OK) rc = precision == IDX_FP32_BULK ? batch_occupancy<float>(b) : batch_occupancy<double>(b);
  if (rc != IDX_OK) {
    idx_batch_destroy(b);
    return rc;
  }
  *out = b;
  return IDX_OK;
}

void idx_batch_destroy(idx_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < kSoloStreams; ++k)
    if (b->side[k]) cudaStreamSynchronize(b->side[k]);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->lists) cudaFree(b->lists);
  if (b->header) cudaFree(b->header);
  if (b->host_gather) cudaFreeHost(b->host_gather);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  for (int k = 0; k < kSoloStreams; ++k) {
    if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
  }
  delete b;
}

int idx_batch_add(idx_batch* b, idx_sim* s, double t_end) {
  if (!b || !s || !(t_end >= 0.0)) return IDX_EINVAL;
  if (s->solver.precision != b->precision || s->device != b->device) return IDX_EINVAL;
  for (idx_sim* m : b->sims)
    if (m == s) return IDX_EINVAL;
  IDX_TRY(cudaStreamSynchronize(b->stream));
  IDX_TRY(cudaStreamSynchronize(s->stream));  // the sim's own work (its state upload) first
  int rc = arm_end_time(b->stream, s, t_end);
  if (rc != IDX_OK) return rc;
  s->w_fresh = false;  // a work-list member's W does not follow its state
  b->sims.push_back(s);
  b->dirty = true;
  return IDX_OK;
}

int idx_batch_remove(idx_batch* b, idx_sim* s) {
  if (!b || !s) return IDX_EINVAL;
  for (size_t i = 0; i < b->sims.size(); ++i) {
    if (b->sims[i] != s) continue;
    IDX_TRY(cudaStreamSynchronize(b->stream));
    b->sims.erase(b->sims.begin() + i);
    b->dirty = true;
    // back to unclamped single-sim stepping
    int rc = arm_end_time(b->stream, s, std::numeric_limits<double>::infinity());
    if (rc != IDX_OK) return rc;
    return IDX_OK;
  }
  return IDX_EINVAL;
}

int idx_batch_step(idx_batch* b, int ncycles) {
  if (!b || ncycles < 0) return IDX_EINVAL;
  if (b->sims.empty() || ncycles == 0) return IDX_OK;
  const bool f32 = b->precision == IDX_FP32_BULK;
  int rc = f32 ? batch_prepare<float>(b) : batch_prepare<double>(b);
  if (rc != IDX_OK) return rc;
  for (int q = 0; q < ncycles; ++q) IDX_TRY(cudaGraphLaunch(b->exec, b->stream));
  return IDX_OK;
}

int idx_batch_poll(idx_batch* b, idx_sim** finished, int cap, int* n_finished, int* n_active) {
  if (!b || (cap > 0 && !finished)) return IDX_EINVAL;
  const bool f32 = b->precision == IDX_FP32_BULK;
  int rc = f32 ? batch_prepare<float>(b) : batch_prepare<double>(b);
  if (rc != IDX_OK) return rc;
  const int n = (int)b->sims.size();
  int nf = 0, na = 0;
  if (n > 0) {
    if (f32) kb_gather<float><<<1, kThreads, 0, b->stream>>>((const BatchDev<float>*)b->header);
    else kb_gather<double><<<1, kThreads, 0, b->stream>>>((const BatchDev<double>*)b->header);
    IDX_TRY(cudaGetLastError());
    BatchDev<double> h;  // only the gather pointer is read; same layout for both types
    IDX_TRY(cudaMemcpyAsync(&h, b->header, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    IDX_TRY(cudaStreamSynchronize(b->stream));
    IDX_TRY(cudaMemcpyAsync(b->host_gather, h.gather, sizeof(Ctrl) * n, cudaMemcpyDeviceToHost, b->stream));
    IDX_TRY(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; ++i) {
      const Ctrl& c = b->host_gather[i];
      idx_sim* s = b->sims[i];
      *s->host_ctrl = c;  // keep the sim's mirror current
      if (c.done || c.err) {
        if (nf < cap) finished[nf] = s;
        ++nf;
      } else {
        ++na;
      }
    }
  }
  if (n_finished) *n_finished = nf;
  if (n_active) *n_active = na;
  return IDX_OK;
}

int idx_batch_shapes(const idx_batch* b, int shapes[3]) {
  if (!b || !shapes) return IDX_EINVAL;
  for (int d = 0; d < 3; ++d) shapes[d] = b->shape[d];
  return IDX_OK;
}

int idx_batch_set_shapes(idx_batch* b, const int shapes[3]) {
  if (!b || !shapes) return IDX_EINVAL;
  for (int d = 0; d < 3; ++d) {
    const int x = shapes[d];
    const bool march = x == 2 || x == 4 || x == 8 || x == 16 || x == 32;
    if (!march && !(x == -1 && d == 0) && !((x == 116 || x == 132) && d != 0)) return IDX_EINVAL;
  }
  IDX_TRY(cudaStreamSynchronize(b->stream));
  for (int d = 0; d < 3; ++d) {
    b->shape[d] = shapes[d];
    b->fallback[d] = kSegDefault;
  }
  b->tuned = true;
  b->dirty = true;  // rebuild the work-lists for the new shapes
  return IDX_OK;
}

}  // extern "C"
