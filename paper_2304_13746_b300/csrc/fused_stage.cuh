// fused_stage.cuh -- one kernel for the reconstruction, Riemann fluxes, E^c edge EMFs and
// update of an RK stage in the FP32-bulk variant (Secs. 2.3, 2.4, 2.7; Eqs. 5, 6, 9, 10).
// Included by idx_stage.cu inside its anonymous namespace, after the per-face and
// per-cell pieces it reuses (vanleer_half, riemann_flux, emf_ec, block_max_to).
//
// The split stage hands the fluxes (8 words per face and direction), the edge EMFs and
// the primitives through HBM between six kernels, and runs the FP64-pipe update after
// the FP32-pipe sweeps.  Here a CTA owns a 32 x 8 tile of the x-y plane and marches it
// through a chunk of z-planes.  A ring of four primitive planes (the tile plus its 2-cell
// periodic halo, FP32, 8 variables) arrives by bulk tensor copies (TMA) into shared
// memory, one plane ahead of use.  Per plane q the CTA forms, in shared memory:
//   * the x-, y- and z-face fluxes of plane q (the z-faces between planes q-1 and q) for
//     the tile and the halo faces its EMFs need -- the one recomputation of this design,
//     +27 % Riemann solves, in the FP32 pipe that has room for them;
//   * the cell-centre EMFs -(v x B) of plane q;
//   * the E^c EMFs of the edges of plane q;
// and then updates the cells of plane q-1 (FP64 accumulation, RK combine) from the
// registers that carry the x/y flux divergence and the lower z-face flux of each column.
// Fluxes and EMFs never touch HBM.  Two CTAs per SM (108.6 KB of shared memory each)
// interleave the FP32 flux phase of one with the FP64 update of the other.
//
// Requirements (checked on the host): FP32 bulk, PLM, field induction, every direction
// integrated, nx % 32 == 0, ny % 8 == 0, nz a multiple of the z-chunk.
#pragma once

namespace fused {

constexpr int TX = 32, TY = 8;           // cells of a tile in x and y
constexpr int NT = TX * TY;              // threads per CTA: one per cell of a plane
// primitive plane in shared memory: 9 boxes (y parts lo 2 / body 8 / hi 2 rows, x parts
// lo 4 / body 32 / hi 4 columns), each [8 variables][rows][columns]
constexpr int WX = 40, WY = 12, NV = 8;
constexpr int WPLANE = NV * WX * WY;     // 3840 floats
constexpr int RING = 4;
// face and edge sets of a plane (index = row * width + column)
constexpr int FXW = TX + 1, FXH = TY + 2;  // x-faces i0..i0+32, rows j0-1..j0+8
constexpr int FYW = TX + 2, FYH = TY + 1;  // y-faces columns i0-1..i0+32, rows j0..j0+8
constexpr int FZW = TX + 2, FZH = TY + 2;  // z-faces columns i0-1..i0+32, rows j0-1..j0+8
constexpr int NFX = FXW * FXH, NFY = FYW * FYH, NFZ = FZW * FZH;  // 330, 306, 340
constexpr int CCW = TX + 2, CCH = TY + 2, NCC = CCW * CCH;        // cells i0-1.., j0-1..
constexpr int EZW = TX + 1, EZH = TY + 1, NEZ = EZW * EZH;        // edges i0..i0+32, j0..j0+8
constexpr int EXW = TX, EXH = TY + 1, NEX = EXW * EXH;            // i0..i0+31, j0..j0+8
constexpr int EYW = TX + 1, EYH = TY, NEY = EYW * EYH;            // i0..i0+32, j0..j0+7

// shared-memory plan, in floats
constexpr int OFF_W = 0;
constexpr int OFF_FX = OFF_W + RING * WPLANE;   // 8 slots x NFX
constexpr int OFF_FY = OFF_FX + 8 * NFX;
constexpr int OFF_FZ = OFF_FY + 8 * NFY;
constexpr int OFF_PX = OFF_FZ + 8 * NFZ;        // plane q-1: x-face mass flux, B_z flux
constexpr int OFF_PY = OFF_PX + 2 * NFX;        // plane q-1: y-face mass flux, B_z flux
constexpr int OFF_CC = OFF_PY + 2 * NFY;        // plane q: cell-centre EMF x, y, z
constexpr int OFF_CP = OFF_CC + 3 * NCC;        // plane q-1: cell-centre EMF x, y
constexpr int OFF_EZ = OFF_CP + 2 * NCC;        // 2 planes (q & 1)
constexpr int OFF_EX = OFF_EZ + 2 * NEZ;
constexpr int OFF_EY = OFF_EX + 2 * NEX;
constexpr int NFLOATS = OFF_EY + 2 * NEY;
constexpr size_t SMEM_BYTES = sizeof(float) * NFLOATS + 8 * RING;  // + the ring's mbarriers
static_assert(OFF_FX * sizeof(float) % 128 == 0, "TMA destinations stay 128-byte aligned");
static_assert(SMEM_BYTES <= 113 * 1024, "two CTAs per SM");

// box geometry of the 9 parts of a primitive plane
__host__ __device__ constexpr int ypart_rows(int yp) { return yp == 1 ? TY : 2; }
__host__ __device__ constexpr int xpart_cols(int xp) { return xp == 1 ? TX : 4; }
__host__ __device__ constexpr int part_offset(int yp, int xp) {
  int off = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      if (a == yp && b == xp) return off;
      off += NV * ypart_rows(a) * xpart_cols(b);
    }
  return off;
}
static_assert(part_offset(2, 2) + NV * 2 * 4 == WPLANE, "plane layout");

// Float offset of cell (row r in 0..11 = j - (j0 - 2), column x in -4..35 = i - i0) of a
// plane buffer, and the stride between its variables.
__device__ __forceinline__ int cell_at(int r, int x, int& vstride) {
  const int yp = r < 2 ? 0 : (r < 2 + TY ? 1 : 2);
  const int rr = r - (yp == 0 ? 0 : (yp == 1 ? 2 : 2 + TY));
  const int xp = x < 0 ? 0 : (x < TX ? 1 : 2);
  const int xx = x - (xp == 0 ? -4 : (xp == 1 ? 0 : TX));
  const int by = ypart_rows(yp), bx = xpart_cols(xp);
  vstride = by * bx;
  // part offsets: a small table folded by the compiler
  int base;
  switch (yp * 3 + xp) {
    case 0: base = part_offset(0, 0); break;
    case 1: base = part_offset(0, 1); break;
    case 2: base = part_offset(0, 2); break;
    case 3: base = part_offset(1, 0); break;
    case 4: base = part_offset(1, 1); break;
    case 5: base = part_offset(1, 2); break;
    case 6: base = part_offset(2, 0); break;
    case 7: base = part_offset(2, 1); break;
    default: base = part_offset(2, 2); break;
  }
  return base + rr * bx + xx;
}

// rotated variable slots (rho, v_n, v_t1, v_t2, P, B_t1, B_t2) of direction d, t1 = d+1
__device__ __forceinline__ int rot_var(int d, int q) {
  // d = 0: 0 1 2 3 4 6 7; d = 1: 0 2 3 1 4 7 5; d = 2: 0 3 1 2 4 5 6
  constexpr int tab[3][7] = {{0, 1, 2, 3, 4, 6, 7}, {0, 2, 3, 1, 4, 7, 5}, {0, 3, 1, 2, 4, 5, 6}};
  return tab[d][q];
}

}  // namespace fused

struct FusedMaps {
  CUtensorMap box[4];  // W boxes {4, 2}, {32, 2}, {4, 8}, {32, 8} x 1 plane x 8 variables
};

// Issue the 9 box copies of primitive plane p (wrapped periodically) of the tile at
// (i0, j0) into plane buffer dst, completing on bar.
__device__ __forceinline__ void fused_load_plane(const Geo& g, const FusedMaps& M, float* dst,
                                                 int i0, int j0, int p, uint64_t* bar) {
  using namespace fused;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  int z = p % nz;
  if (z < 0) z += nz;
  mbar_arrive_expect_tx(bar, (uint32_t)(WPLANE * sizeof(float)));
  const int ys[3] = {j0 - 2 < 0 ? j0 - 2 + ny : j0 - 2, j0, j0 + TY >= ny ? j0 + TY - ny : j0 + TY};
  const int xs[3] = {i0 - 4 < 0 ? i0 - 4 + nx : i0 - 4, i0, i0 + TX >= nx ? i0 + TX - nx : i0 + TX};
#pragma unroll
  for (int yp = 0; yp < 3; ++yp)
#pragma unroll
    for (int xp = 0; xp < 3; ++xp) {
      const int m = (yp == 1 ? 2 : 0) + (xp == 1 ? 1 : 0);
      tma_load_4d(dst + part_offset(yp, xp), &M.box[m], xs[xp], ys[yp], z, 0, bar);
    }
}

// One face of direction d: reconstruct from the 4 cells along d (offsets c[0..3] into the
// plane buffers P[0..3], variable strides s[0..3]) and solve the Riemann problem.
__device__ __forceinline__ void fused_face(const Geo& g, int d, const float* const P[4],
                                           const int c[4], const int s[4], float bn,
                                           float* out, int nface) {
  float w[4][7];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int q = 0; q < 7; ++q) w[k][q] = P[k][c[k] + fused::rot_var(d, q) * s[k]];
  float sl[7], sr[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    sl[q] = vanleer_half(w[1][q] - w[0][q], w[2][q] - w[1][q]);  // cell f-1, toward face f
    sr[q] = vanleer_half(w[2][q] - w[1][q], w[3][q] - w[2][q]);  // cell f, away from face f
  }
  Side<float> L, R;
  L.r = w[1][0] + sl[0]; R.r = w[2][0] - sr[0];
  L.u = w[1][1] + sl[1]; R.u = w[2][1] - sr[1];
  L.v = w[1][2] + sl[2]; R.v = w[2][2] - sr[2];
  L.w = w[1][3] + sl[3]; R.w = w[2][3] - sr[3];
  L.p = w[1][4] + sl[4]; R.p = w[2][4] - sr[4];
  L.b1 = w[1][5] + sl[5]; R.b1 = w[2][5] - sr[5];
  L.b2 = w[1][6] + sl[6]; R.b2 = w[2][6] - sr[6];
  float flux[7], cmax;
  riemann_flux(g.riemann, L, R, bn, g.gammaf, g.gm1invf, flux, cmax);
#pragma unroll
  for (int q = 0; q < 7; ++q) out[q * nface] = flux[q];
  out[7 * nface] = cmax;
}

template <bool COMBINE>
__global__ void __launch_bounds__(fused::NT, 2)
    k_stage_fused(Geo g, const __grid_constant__ FusedMaps M, const double* bx_face,
                  const double* by_face, const double* bz_face, Ptr8<const double> Uin,
                  Ptr8<const double> U0, Ptr8<double> Uout, Ctrl* ctrl, int zchunk, double w,
                  double w0, double dt_fixed) {
  using namespace fused;
  // dt_fixed > 0: a timing launch outside a cycle (the autotuner), which writes only Uout
  const double dt = dt_fixed > 0.0 ? dt_fixed : ctrl->dt;
  if (!(dt > 0.0)) return;
  extern __shared__ __align__(128) unsigned char fsm_raw[];
  float* sm = reinterpret_cast<float*>(fsm_raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(fsm_raw + sizeof(float) * NFLOATS);
  const int tid = threadIdx.x;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  int b = blockIdx.x;
  const int ntx = nx / TX, nty = ny / TY;
  const int i0 = (b % ntx) * TX;
  b /= ntx;
  const int j0 = (b % nty) * TY;
  const int k0 = (b / nty) * zchunk;
  const int k1 = k0 + zchunk;                 // planes k0 .. k1-1 are updated here
  const int pfirst = k0 - 2;                  // first primitive plane the CTA loads
  auto slot_of = [&](int p) { return (p - pfirst) & (RING - 1); };
  auto parity_of = [&](int p) { return (uint32_t)(((p - pfirst) >> 2) & 1); };
  float* Wr = sm + OFF_W;
  const float idx = g.inv_dlf[0], idy = g.inv_dlf[1], idz = g.inv_dlf[2];

  if (tid == 0) {
    for (int r = 0; r < RING; ++r) mbar_init(&bar[r], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    for (int p = pfirst; p < pfirst + RING; ++p)
      fused_load_plane(g, M, Wr + slot_of(p) * WPLANE, i0, j0, p, &bar[slot_of(p)]);
  int issued = pfirst + RING - 1;             // planes up to this one have been requested
  int landed = pfirst - 1;                    // planes up to this one have landed
  bool ok = true;

  // carried per column (cell i0 + tx, j0 + ty): x/y divergence and speeds of plane q-1,
  // the lower z-face flux of plane q-1
  const int tx = tid % TX, ty = tid / TX;
  float dxy[5] = {0, 0, 0, 0, 0}, cxy = 0.f, fzl[5] = {0, 0, 0, 0, 0}, czl = 0.f;
  float inv_max = 0.f;
  const float dtf = d2f_warp(dt);
  const float wdt = d2f_warp(w * dt);
  const bool same_w = w == w0;

  for (int q = k0 - 1; q <= k1; ++q) {
    // wait for the planes this iteration reads: q (in-plane sweeps) and q-2 .. q+1 (z)
    const int need = (q == k0 - 1) ? q : q + 1;
    while (ok && landed < need) {
      if (mbar_wait(&bar[slot_of(landed + 1)], parity_of(landed + 1), kWaitNs)) ++landed;
      else ok = false;
    }
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    const float* Pq = Wr + slot_of(q) * WPLANE;
    float* FX = sm + OFF_FX;
    float* FY = sm + OFF_FY;
    float* FZ = sm + OFF_FZ;
    float* CC = sm + OFF_CC;
    const bool zfaces = q >= k0;              // F_z(q) needs planes q-2 .. q+1
    // ---- fluxes of plane q: x-faces, y-faces, z-faces in one list
    const int nall = NFX + NFY + (zfaces ? NFZ : 0);
    const int zq = q < 0 ? q + nz : (q >= nz ? q - nz : q);
    for (int f = tid; f < nall; f += NT) {
      const float* P[4];
      int c[4], s[4];
      if (f < NFX) {
        const int fx = f % FXW, fy = f / FXW;   // face i0 + fx, row j0 - 1 + fy
        for (int k = 0; k < 4; ++k) {
          P[k] = Pq;
          c[k] = fused::cell_at(fy + 1, fx - 2 + k, s[k]);
        }
        int i = i0 + fx, j = j0 - 1 + fy;
        if (i >= nx) i -= nx;
        if (j < 0) j += ny;
        if (j >= ny) j -= ny;
        const float bn = to_bulk<float>(bx_face[i + nx * (j + ny * zq)]);
        fused_face(g, 0, P, c, s, bn, FX + f, NFX);
      } else if (f < NFX + NFY) {
        const int e = f - NFX;
        const int fx = e % FYW, fy = e / FYW;   // column i0 - 1 + fx, face j0 + fy
        for (int k = 0; k < 4; ++k) {
          P[k] = Pq;
          c[k] = fused::cell_at(fy + k, fx - 1, s[k]);
        }
        int i = i0 - 1 + fx, j = j0 + fy;
        if (i < 0) i += nx;
        if (i >= nx) i -= nx;
        if (j >= ny) j -= ny;
        const float bn = to_bulk<float>(by_face[i + nx * (j + ny * zq)]);
        fused_face(g, 1, P, c, s, bn, FY + e, NFY);
      } else {
        const int e = f - NFX - NFY;
        const int fx = e % FZW, fy = e / FZW;   // column i0 - 1 + fx, row j0 - 1 + fy
        for (int k = 0; k < 4; ++k) {
          P[k] = Wr + slot_of(q - 2 + k) * WPLANE;
          c[k] = fused::cell_at(fy + 1, fx - 1, s[k]);
        }
        int i = i0 - 1 + fx, j = j0 - 1 + fy;
        if (i < 0) i += nx;
        if (i >= nx) i -= nx;
        if (j < 0) j += ny;
        if (j >= ny) j -= ny;
        const float bn = to_bulk<float>(bz_face[i + nx * (j + ny * zq)]);
        fused_face(g, 2, P, c, s, bn, FZ + e, NFZ);
      }
    }
    // cell-centre EMFs -(v x B_c) of plane q, cells i0-1 .. i0+32, j0-1 .. j0+8
    for (int e = tid; e < NCC; e += NT) {
      const int cx = e % CCW, cy = e / CCW;
      int sv;
      const int o = fused::cell_at(cy + 1, cx - 1, sv);
      const float vx = Pq[o + 1 * sv], vy = Pq[o + 2 * sv], vz = Pq[o + 3 * sv];
      const float bxc = Pq[o + 5 * sv], byc = Pq[o + 6 * sv], bzc = Pq[o + 7 * sv];
      CC[e] = -(vy * bzc - vz * byc);
      CC[NCC + e] = -(vz * bxc - vx * bzc);
      CC[2 * NCC + e] = -(vx * byc - vy * bxc);
    }
    __syncthreads();
    // the ring slot of plane q-2 is free now: fetch plane q+2 into it
    if (zfaces && q + 2 <= k1 + 1) {
      if (tid == 0) {
        fence_proxy_async();
        fused_load_plane(g, M, Wr + slot_of(q + 2) * WPLANE, i0, j0, q + 2, &bar[slot_of(q + 2)]);
      }
      issued = q + 2;
    }
    // x/y divergence and speeds of this column at plane q (for its update next iteration);
    // slots of the conserved fields rho, m_x, m_y, m_z, E in each direction's flux order
    float dxy_q[5], cxy_q;
    {
      constexpr int sx[5] = {0, 1, 2, 3, 4}, sy[5] = {0, 3, 1, 2, 4};
      const int fxa = (ty + 1) * FXW + tx, fxb = fxa + 1;          // x-faces i, i+1 of row j
      const int fya = ty * FYW + tx + 1, fyb = fya + FYW;          // y-faces j, j+1 of column i
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        float dv = 0.f;
        dv += (FX[sx[k] * NFX + fxb] - FX[sx[k] * NFX + fxa]) * idx;
        dv += (FY[sy[k] * NFY + fyb] - FY[sy[k] * NFY + fya]) * idy;
        dxy_q[k] = dv;
      }
      float iv = 0.f;
      iv += max_nn(FX[7 * NFX + fxa], FX[7 * NFX + fxb]) * idx;
      iv += max_nn(FY[7 * NFY + fya], FY[7 * NFY + fyb]) * idy;
      cxy_q = iv;
    }
    // ---- E^c EMFs of plane q (edges at the lower x/y/z faces of the cells of plane q)
    const int pe = q & 1, po = pe ^ 1;       // EMF ring slots of planes q and q-1
    float* EZ = sm + OFF_EZ + pe * NEZ;
    float* EX = sm + OFF_EX + pe * NEX;
    float* EY = sm + OFF_EY + pe * NEY;
    const float* PX = sm + OFF_PX;
    const float* PY = sm + OFF_PY;
    const float* CP = sm + OFF_CP;
    if (zfaces) {
      const int nz_e = (q < k1) ? NEZ : 0;    // E_z of plane k1 is not used
      const int nedge = nz_e + NEX + NEY;
      for (int e = tid; e < nedge; e += NT) {
        if (e < nz_e) {                         // E_z: a = x, b = y
          const int ex = e % EZW, ey = e / EZW;
          const int xa0 = (ey + 1) * FXW + ex, xa1 = ey * FXW + ex;         // (i, j), (i, j-1)
          const int yb0 = ey * FYW + ex + 1, yb1 = ey * FYW + ex;           // (i, j), (i-1, j)
          const int c00 = (ey + 1) * CCW + ex + 1, c01 = ey * CCW + ex + 1;
          const int c10 = (ey + 1) * CCW + ex, c11 = ey * CCW + ex;
          const float* C = CC + 2 * NCC;
          EZ[e] = emf_ec(-FX[5 * NFX + xa0], -FX[5 * NFX + xa1], FY[6 * NFY + yb0],
                         FY[6 * NFY + yb1], C[c00], C[c01], C[c10], C[c11], FX[xa0], FX[xa1],
                         FY[yb0], FY[yb1]);
        } else if (e < nz_e + NEX) {            // E_x: a = y, b = z
          const int h = e - nz_e;
          const int ex = h % EXW, ey = h / EXW;
          const int ya = ey * FYW + ex + 1;                                 // (i, j) both planes
          const int zb0 = (ey + 1) * FZW + ex + 1, zb1 = ey * FZW + ex + 1;  // (i, j), (i, j-1)
          const int c0 = (ey + 1) * CCW + ex + 1, c1 = ey * CCW + ex + 1;   // (i, j), (i, j-1)
          EX[h] = emf_ec(-FY[5 * NFY + ya], -PY[NFY + ya], FZ[6 * NFZ + zb0], FZ[6 * NFZ + zb1],
                         CC[c0], CP[c0], CC[c1], CP[c1], FY[ya], PY[ya], FZ[zb0], FZ[zb1]);
        } else {                                // E_y: a = z, b = x
          const int h = e - nz_e - NEX;
          const int ex = h % EYW, ey = h / EYW;
          const int za0 = (ey + 1) * FZW + ex + 1, za1 = (ey + 1) * FZW + ex;  // (i, j), (i-1, j)
          const int xb = (ey + 1) * FXW + ex;                                // (i, j) both planes
          const int c0 = (ey + 1) * CCW + ex + 1, c1 = (ey + 1) * CCW + ex;  // (i, j), (i-1, j)
          EY[h] = emf_ec(-FZ[5 * NFZ + za0], -FZ[5 * NFZ + za1], FX[6 * NFX + xb], PX[NFX + xb],
                         CC[NCC + c0], CC[NCC + c1], CP[NCC + c0], CP[NCC + c1], FZ[za0],
                         FZ[za1], FX[xb], PX[xb]);
        }
      }
    }
    __syncthreads();
    // ---- update of plane q-1 (its upper z-face flux and upper EMFs are those of plane q)
    const int fzc = (ty + 1) * FZW + tx + 1;  // this column's z-face in the plane buffers
    float fzh[5] = {0, 0, 0, 0, 0}, czh = 0.f;
    if (zfaces) {
      constexpr int sz[5] = {0, 2, 3, 1, 4};
#pragma unroll
      for (int k = 0; k < 5; ++k) fzh[k] = FZ[sz[k] * NFZ + fzc];
      czh = FZ[7 * NFZ + fzc];
    }
    if (q - 1 >= k0 && q - 1 < k1) {
      const int k = q - 1;
      const int i = i0 + tx, j = j0 + ty;
      const long c = i + (long)nx * (j + (long)ny * k);
      const float* EZo = sm + OFF_EZ + po * NEZ;
      const float* EXo = sm + OFF_EX + po * NEX;
      const float* EYo = sm + OFF_EY + po * NEY;
      double out[8];
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const float dv = dxy[f] + (fzh[f] - fzl[f]) * idz;
        if (COMBINE) {
          if (same_w) out[f] = fma(w, U0.f[f][c] + Uin.f[f][c], f2d_warp(-wdt * dv));
          else out[f] = fma(w0, U0.f[f][c], w * Uin.f[f][c]) + f2d_warp(-wdt * dv);
        } else {
          out[f] = Uin.f[f][c] + f2d_warp(-dtf * dv);
        }
      }
      // face fields: B -= dt curl E (Eq. 6); E_z of plane k at (i,j), (i+1,j), (i,j+1); E_x,
      // E_y of planes k and k+1
      const float ez00 = EZo[ty * EZW + tx], ez10 = EZo[ty * EZW + tx + 1];
      const float ez01 = EZo[(ty + 1) * EZW + tx];
      const float ex0 = EXo[ty * EXW + tx], ex0y = EXo[(ty + 1) * EXW + tx];
      const float ex1 = EX[ty * EXW + tx];
      const float ey0 = EYo[ty * EYW + tx], ey0x = EYo[ty * EYW + tx + 1];
      const float ey1 = EY[ty * EYW + tx];
      float curl[3];
      curl[0] = 0.f;
      curl[0] += (ez01 - ez00) * idy;
      curl[0] -= (ey1 - ey0) * idz;
      curl[1] = 0.f;
      curl[1] += (ex1 - ex0) * idz;
      curl[1] -= (ez10 - ez00) * idx;
      curl[2] = 0.f;
      curl[2] += (ey0x - ey0) * idx;
      curl[2] -= (ex0y - ex0) * idy;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int f = 5 + m;
        if (COMBINE) {
          if (same_w) out[f] = fma(w, U0.f[f][c] + Uin.f[f][c], f2d_warp(-wdt * curl[m]));
          else out[f] = fma(w0, U0.f[f][c], w * Uin.f[f][c]) + f2d_warp(-wdt * curl[m]);
        } else {
          out[f] = Uin.f[f][c] + f2d_warp(-dtf * curl[m]);
        }
      }
#pragma unroll
      for (int f = 0; f < 8; ++f) Uout.f[f][c] = out[f];
      float iv = cxy;
      iv += max_nn(czl, czh) * idz;
      inv_max = max_nn(inv_max, iv);
    }
    // plane q's EMF inputs become plane q-1's for the next iteration
    for (int e = tid; e < NFX; e += NT) {
      float* PXw = sm + OFF_PX;
      PXw[e] = FX[e];
      PXw[NFX + e] = FX[6 * NFX + e];
    }
    for (int e = tid; e < NFY; e += NT) {
      float* PYw = sm + OFF_PY;
      PYw[e] = FY[e];
      PYw[NFY + e] = FY[5 * NFY + e];
    }
    for (int e = tid; e < NCC; e += NT) {
      float* CPw = sm + OFF_CP;
      CPw[e] = CC[e];
      CPw[NCC + e] = CC[NCC + e];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      dxy[k] = dxy_q[k];
      fzl[k] = fzh[k];
    }
    cxy = cxy_q;
    czl = czh;
    __syncthreads();  // every read of this plane's buffers is done before they are refilled
  }
  if (!ok) {
    // a copy did not land in time: record it, and give every copy still in flight (planes
    // landed+1 .. issued, at most the ring) a bounded time to land before the CTA leaves
    if (tid == 0) flag_timeout(ctrl);
    for (int p = landed + 1; p <= issued; ++p) mbar_wait(&bar[slot_of(p)], parity_of(p), kWaitNs);
    return;
  }
  block_max_to(&ctrl->inv_acc, inv_max);
}
