/*
 * oracle.h -- C interface of the FP64 CPU oracle for one RK2 cycle of ideal MHD.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Method (IDEFIX paper, Lesur et al. 2023):
 *   Eq. (1)-(4)  ideal-MHD conservation laws (no 4*pi in the units),
 *   Eq. (5)      Godunov finite-volume form,
 *   Sec. 2.3     reconstruction on primitives (PLM with van Leer, or the compact
 *                third-order LimO3), HLLD / HLL / Rusanov Riemann solvers,
 *                pressure kept inside the momentum flux,
 *   Sec. 2.4     constrained transport on face-centred B, E^c edge EMF (Eq. 6),
 *   Sec. 2.7     method-of-lines RK2 (Eq. 9, Table 1) and the CFL time step (Eq. 10).
 *
 * Layout: every field is double[nz][ny][nx] (x fastest), periodic in all three
 * directions.  Conserved set: rho, mx, my, mz, E (cell averages) and Bx, By, Bz
 * (face averages: Bx[k][j][i] sits on the x-face at i-1/2, By on the y-face at
 * j-1/2, Bz on the z-face at k-1/2).  A direction with n_d == 1 is not integrated.
 *
 * Return codes: 0 ok; ORA_EINVAL bad argument; ORA_ENONPHYS rho<=0, P<=0 or a
 * non-finite value found while recovering primitives (the flat cell index is
 * written to *bad_cell when the pointer is given).
 */
#ifndef IDX_ORACLE_H
#define IDX_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define ORA_OK 0
#define ORA_EINVAL (-1)
#define ORA_ENONPHYS (-3)

typedef struct {
  int nx, ny, nz;      /* cells per direction, >= 1 */
  double lx, ly, lz;   /* box lengths; cell size = l/n */
} ora_grid;

/* Primitive input (rho, vx, vy, vz, P at cell centres; Bx, By, Bz on faces)
 * -> conserved (rho, mx, my, mz, E, Bx, By, Bz).  E uses the face-averaged
 * cell-centre B, exactly as primitive recovery inverts it. */
int ora_cons_from_prims(const ora_grid* g, double gamma, const double* const prim[8],
                        double* const cons[8]);

/* Conserved -> primitives (rho, vx, vy, vz, P, Bcx, Bcy, Bcz), all cell-centred. */
int ora_prims(const ora_grid* g, double gamma, const double* const cons[8], double* const w[8],
              long* bad_cell);

/* van Leer limited slope of one variable from the values at i-1, i, i+1. */
double ora_vanleer(double wm, double w0, double wp);

/* LimO3 face value (Sec. 2.3, the compact third-order scheme of Cada & Torrilhon 2009) of a
 * cell with value w0 on its side toward w_face, w_back the neighbour on the other side. */
double ora_limo3_face(double w_back, double w0, double w_face);

/* HLLD flux at one interface whose normal is "x".  wL, wR = (rho, u, v, w, P, Bt1, Bt2);
 * bn = normal field.  F = fluxes of (rho, m_n, m_t1, m_t2, E, Bt1, Bt2).  sL, sR = the
 * outer wave-speed estimates. */
int ora_hlld(const double wL[7], const double wR[7], double bn, double gamma, double F[7],
             double* sL, double* sR);

/* Any of the Riemann solvers of Sec. 2.3 that the build covers: solver 1 Rusanov
 * (Lax-Friedrichs), 2 HLL, 4 HLLD; same arguments as ora_hlld.  All three report the
 * HLLD outer speed estimates in sL, sR (the CFL condition does not depend on the solver). */
int ora_riemann(int solver, const double wL[7], const double wR[7], double bn, double gamma,
                double F[7], double* sL, double* sR);

/* ora_cycle with a chosen Riemann solver (1, 2 or 4). */
int ora_cycle_solver(const ora_grid* g, double gamma, double cfl, int solver, double* const u[8],
                     double* inv_dt, double dt_max, double* dt_taken, long* bad_cell);

/* One cycle with a chosen solver (1, 2, 4) and RK order (2 or 3, Table 1). */
int ora_cycle_rk(const ora_grid* g, double gamma, double cfl, int solver, int rk_order,
                 double* const u[8], double* inv_dt, double dt_max, double* dt_taken,
                 long* bad_cell);

/* Face field from an edge vector potential (Sec. 2.4, Eq. 8, discrete Stokes on each
 * face): B_d = bmean_d + curl_d A.  A[e] is stored like the edge EMF E_e (at the cell
 * whose lower (e+1)- and (e+2)-faces bound the edge); differences along a direction with
 * one cell are dropped. */
int ora_b_from_potential(const ora_grid* g, const double* const A[3], const double bmean[3],
                         double* const B[3]);

/* One cycle with the vector-potential induction (Sec. 2.4, Eqs. 7-8): every stage steps
 * A on the edges with -E (RK weights of Table 1) and sets the face field of u to
 * Bref + curl A.  u (8 fields) and A (3 edge fields) in/out; Bref (3 face fields) in. */
int ora_cycle_vp(const ora_grid* g, double gamma, double cfl, int solver, int rk_order,
                 double* const u[8], double* const A[3], const double* const Bref[3],
                 double* inv_dt, double dt_max, double* dt_taken, long* bad_cell);

/* Ideal-MHD physical flux along "x" of one state (same ordering as ora_hlld). */
int ora_phys_flux(const double w[7], double bn, double gamma, double F[7]);

/* E^c edge EMF of Gardiner & Stone (2005) for one edge, generic first/second directions
 * a, b: X[r] a-face EMFs at b-index J (r=0) and J-1 (r=1); Y[c] b-face EMFs at a-index
 * I (c=0) and I-1 (c=1); C[c][r] cell-centre EMFs; Fa[r], Fb[c] the matching mass
 * fluxes; da, db cell sizes. */
double ora_emf_ec(const double X[2], const double Y[2], const double C[2][2], const double Fa[2],
                  const double Fb[2], double da, double db);

/* Signal-speed-only pass on a state: returns max over cells of
 * sum_d max(c_face(i-1/2), c_face(i+1/2)) / dl_d  (the inverse CFL time). */
int ora_speed_pass(const ora_grid* g, double gamma, const double* const cons[8], double* inv_dt,
                   long* bad_cell);

/* ora_speed_pass with a chosen reconstruction: recon 1 PLM (van Leer), 3 LimO3. */
int ora_speed_pass_recon(const ora_grid* g, double gamma, int recon, const double* const cons[8],
                         double* inv_dt, long* bad_cell);

/* ora_stage with a chosen reconstruction (1, 3) and Riemann solver (1, 2, 4). */
int ora_stage_scheme(const ora_grid* g, double gamma, double dt, int recon, int solver,
                     const double* const uin[8], const double* const u0[8], double w, double w0,
                     double* const uout[8], double* inv_dt, long* bad_cell);

/* One cycle with every choice: reconstruction (1 PLM, 3 LimO3), Riemann solver (1, 2, 4),
 * RK order (2, 3) and induction form (A and Bref both NULL: face field stepped; both given:
 * vector potential as in ora_cycle_vp). */
int ora_cycle_scheme(const ora_grid* g, double gamma, double cfl, int recon, int solver,
                     int rk_order, double* const u[8], double* const A[3],
                     const double* const Bref[3], double* inv_dt, double dt_max,
                     double* dt_taken, long* bad_cell);

/* One stage: uout = w * S_dt(uin) + w0 * u0 (u0 may be NULL when w0 == 0).
 * *inv_dt receives the stage's inverse CFL time. */
int ora_stage(const ora_grid* g, double gamma, double dt, const double* const uin[8],
              const double* const u0[8], double w, double w0, double* const uout[8],
              double* inv_dt, long* bad_cell);

/* One RK2 cycle in place.  dt = min(cfl / *inv_dt, dt_max); on return *inv_dt holds
 * max(inv of stage 1, inv of stage 2), the input of the next cycle's dt. */
int ora_cycle(const ora_grid* g, double gamma, double cfl, double* const u[8], double* inv_dt,
              double dt_max, double* dt_taken, long* bad_cell);

/* Operation count of one RK2 cycle on the given state, per cell-update:
 * counts[0] add/sub, [1] mul, [2] div, [3] sqrt, [4] compare.  Every add/sub, mul, div
 * and square root of the oracle's own arithmetic counts once (it has no fused operations);
 * negation and absolute value do not count. */
int ora_count_cycle(const ora_grid* g, double gamma, double cfl, const double* const u[8],
                    double inv_dt, double counts[5]);

/* Parts of the method the counts are split into (ora_count_cycle_parts). */
enum {
  ORA_PART_PRIMS = 0,    /* primitive recovery, Sec. 2.1 definitions                    */
  ORA_PART_SLOPE = 1,    /* van Leer slopes; formed here for both faces that use a cell  */
  ORA_PART_FACE = 2,     /* face values w +- slope/2 (or LimO3 face values)              */
  ORA_PART_RIEMANN = 3,  /* Riemann solver per face, Sec. 2.3                            */
  ORA_PART_SPEED = 4,    /* face signal speed max(|S_L|, |S_R|), Eq. 10                  */
  ORA_PART_INVDT = 5,    /* inverse CFL time per cell and its maximum, Eq. 10            */
  ORA_PART_CELL_EMF = 6, /* cell-centre EMF -(v x B); formed here at all 4 edges of a cell */
  ORA_PART_EDGE = 7,     /* E^c edge EMF from face and cell-centre EMFs, Sec. 2.4        */
  ORA_PART_DIFF = 8,     /* flux differences and EMF curls over the cell size, Eqs. 5-6  */
  ORA_PART_ACCUM = 9,    /* U* = U - dt (difference): the accumulation into the state    */
  ORA_PART_COMBINE = 10, /* RK weights w U* + w0 U0, Eq. 9                               */
  ORA_PART_DT = 11,      /* dt = cfl / inv and the max over stages, Eq. 10               */
  ORA_PART_POTENTIAL = 12, /* vector-potential step and curl, Eqs. 7-8                   */
  ORA_NUM_PARTS = 13
};

/* ora_count_cycle split by part: counts[5 * part + k], k as in ora_count_cycle. */
int ora_count_cycle_parts(const ora_grid* g, double gamma, double cfl, const double* const u[8],
                          double inv_dt, double counts[5 * ORA_NUM_PARTS]);

/* Operation counts of single calls of the oracle's pieces, for hand-counted pins:
 * one van Leer slope, one total energy and physical flux (Eq. 1 fluxes), one HLLD
 * solve and one E^c edge EMF.  counts as in ora_count_cycle. */
int ora_count_vanleer(double wm, double w0, double wp, double counts[5]);
int ora_count_energy_flux(const double w[7], double bn, double gamma, double counts_energy[5],
                          double counts_flux[5]);
int ora_count_hlld(const double wL[7], const double wR[7], double bn, double gamma,
                   double counts[5]);
int ora_count_emf_ec(const double X[2], const double Y[2], const double C[2][2],
                     const double Fa[2], const double Fb[2], double da, double db,
                     double counts[5]);

/* Operation counts per face of direction d (0, 1, 2) on the given state, split into the
 * HLLD solve and the reconstruction of the two face states (which evaluates the slope of
 * both adjacent cells): [0] add/sub, [1] mul, [2] div, [3] sqrt, [4] compare. */
int ora_count_faces(const ora_grid* g, double gamma, const double* const u[8], int d,
                    double counts_hlld[5], double counts_recon[5]);

/* The same per-face counts split three ways: counts[0..4] the HLLD solve, [5..9] the van
 * Leer slopes of both face states (each cell's slope is formed for both of its faces),
 * [10..14] the face values w +- slope / 2. */
int ora_count_faces_parts(const ora_grid* g, double gamma, const double* const u[8], int d,
                          double counts[15]);

/* Number of host threads the oracle uses (OpenMP), for reporting. */
int ora_threads(void);

#ifdef __cplusplus
}
#endif
#endif
