/*
 * FP64 CPU oracle for the coupled immersed-boundary lattice-Boltzmann (IB-LB) step of
 * arXiv:2305.18919, "A sharp interface approach for wetting dynamics of coated droplets
 * and soft particles", Sec. III.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, deliberately unoptimised restatement
 * of the method in double precision with plain loops. Only the test-suite, the smoke
 * check and the timed CPU baseline of the benchmark may load it. The CUDA library never
 * links, loads or calls it, and the two share no code, headers or tables.
 *
 * Readings taken where the paper is silent, ambiguous or garbled:
 *  R1  Eq. 10 prints the second-order equilibrium term over 2 c_s^2; it is read as the
 *      standard Hermite term over 2 c_s^4, the only form that gives the viscosity
 *      mu = c_s^2 rho (tau - 1/2) stated in Sec. III.
 *  R2  Eq. 15 prints the first branch of phi_4 as "0 <= |x|" and writes 4x^2 in the second;
 *      read as Peskin's 4-point function: branch 1 for |r| <= 1, branch 2 for 1 <= |r| <= 2.
 *  R3  D3Q19 ordering (the paper gives only the weights): 0 rest, 1..6 = +-x, +-y, +-z,
 *      7..18 the twelve edge diagonals, opposite directions in pairs (2k-1, 2k).
 *  R4  I1, I2 are the Skalak invariants of the in-plane deformation of each face:
 *      I1 = tr(G0^-1 G) - 2 = l1^2 + l2^2 - 2, I2 = det G / det G0 - 1 = l1^2 l2^2 - 1,
 *      G, G0 the current and reference metric of the face's edge vectors.
 *  R5  Eq. 2 is energy per reference area; face energy = A0 * w_S (constant-strain
 *      triangles, first-order finite elements); w_S0 is constant and dropped.
 *  R6  The wall displacement d in Eq. 19 points from the foot point on the wall plane
 *      to the face centroid; the face force is given in equal thirds to its vertices.
 *      No cut-off is applied.
 *  R7  Layers z=0 and z=nz-1 are solid wall nodes; half-way bounce-back planes sit at
 *      z=0.5 and z=nz-1.5. A moving wall adds -2 w_i rho0 (c_i . u_w)/c_s^2 (rho_w=rho0).
 *      Delta-stencil nodes on a wall layer carry the wall velocity when interpolating and
 *      drop force when spreading; nodes outside the array are skipped.
 *  R8  The velocity interpolated to the vertices uses the populations after streaming and
 *      the force field that was spread and used in the same step's collision.
 *  R9  Vertex positions are unwrapped; stencil indices wrap in the periodic directions.
 *
 * Threads: built with OpenMP, the three per-node loops of a step (collision, streaming, the
 * velocity moments) are split over z-planes. Every node's arithmetic is the same as in one
 * thread and no two threads write the same value (streaming's destinations are distinct), so
 * the results are identical for any thread count. Forces, spreading, interpolation and every
 * reduction stay in one thread, in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
static const double CS2 = 1.0 / 3.0;  /* c_s^2 with dx = dt = 1, Sec. III */
static const double INV_CS2 = 3.0;     /* 1 / c_s^2 */

/* R3: D3Q19 velocity set. */
static const int CVEL[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};

/* Weights, Sec. III footnote: 1/3 rest, 1/18 axis, 1/36 diagonal. */
static const double WEIGHT[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static double weight(int i) { return WEIGHT[i]; }

static int opposite(int i) { return i == 0 ? 0 : ((i % 2 == 1) ? i + 1 : i - 1); }

static int wrap(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double *a, const double *b, double *out) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Copy of the velocity table and weights, for the tests that pin them. */
void iblbref_lattice_table(int32_t *c_out /*[19][3]*/, double *w_out /*[19]*/, int32_t *opp_out /*[19]*/) {
  for (int i = 0; i < Q; i++) {
    for (int k = 0; k < 3; k++) c_out[3 * i + k] = CVEL[i][k];
    w_out[i] = weight(i);
    opp_out[i] = opposite(i);
  }
}

/* Eq. 10 with reading R1: f_i^eq = w_i rho [1 + c.u/cs2 + ((c.u)^2 - cs2 u.u)/(2 cs2^2)]. */
void iblbref_equilibrium(double rho, const double *u, double *feq) {
  double uu = dot3(u, u);
  for (int i = 0; i < Q; i++) {
    double c[3] = {CVEL[i][0], CVEL[i][1], CVEL[i][2]};
    double cu = dot3(c, u);
    feq[i] = weight(i) * rho * (1.0 + cu * INV_CS2 + (cu * cu - CS2 * uu) * (0.5 * INV_CS2 * INV_CS2));
  }
}

/* Eq. 9, last term (Guo forcing): w_i (1 - 1/(2 tau)) [(c_i - u).F/cs2 + (c_i.F)(c_i.u)/cs2^2]. */
void iblbref_guo_source(double tau, const double *u, const double *F, double *S) {
  for (int i = 0; i < Q; i++) {
    double c[3] = {CVEL[i][0], CVEL[i][1], CVEL[i][2]};
    double cmu[3] = {c[0] - u[0], c[1] - u[1], c[2] - u[2]};
    S[i] = weight(i) * (1.0 - 0.5 / tau) *
           (dot3(cmu, F) * INV_CS2 + dot3(c, F) * dot3(c, u) * (INV_CS2 * INV_CS2));
  }
}

/* Density and Guo-shifted velocity, Sec. III: rho = sum f, rho u = sum c f + F/2. */
void iblbref_moments(const double *f, const double *F, double *rho_out, double *u_out) {
  double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; i++) {
    rho += f[i];
    for (int k = 0; k < 3; k++) m[k] += CVEL[i][k] * f[i];
  }
  *rho_out = rho;
  for (int k = 0; k < 3; k++) u_out[k] = (m[k] + 0.5 * F[k]) / rho;
}

/* Eq. 9, right-hand side: BGK relaxation towards Eq. 10 plus the Guo source. */
void iblbref_collide_node(double tau, const double *f, const double *F, double *fout) {
  double rho, u[3], feq[Q], S[Q];
  iblbref_moments(f, F, &rho, u);
  iblbref_equilibrium(rho, u, feq);
  iblbref_guo_source(tau, u, F, S);
  double omega = 1.0 / tau;
  for (int i = 0; i < Q; i++) fout[i] = f[i] - omega * (f[i] - feq[i]) + S[i];
}

/* Eq. 15 with reading R2: Peskin's 4-point regularised delta profile. */
double iblbref_phi4(double r) {
  double a = fabs(r);
  if (a <= 1.0) return 0.125 * (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a));
  if (a <= 2.0) return 0.125 * (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a));
  return 0.0;
}

/* ------------------------------------------------------------------------------------ */
/* Interface forces, Eqs. 2 and 16-19.                                                  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  double alpha[3];
  double kV;
  double eps, xi;
  int wall_on, volume_on;
} ref_iface;

typedef struct {
  int has_walls;
  double z_bottom, z_top; /* wall planes */
} ref_walls;

/* Energy of one face (R4, R5) and its gradient with respect to the three vertices. */
static double face_strain_energy(const double *x0, const double *x1, const double *x2,
                                 const double *X0, const double *X1, const double *X2,
                                 const double *alpha, double *g0, double *g1, double *g2) {
  double a[3], b[3], a0[3], b0[3];
  for (int k = 0; k < 3; k++) {
    a[k] = x1[k] - x0[k];
    b[k] = x2[k] - x0[k];
    a0[k] = X1[k] - X0[k];
    b0[k] = X2[k] - X0[k];
  }
  /* reference metric G0 and its inverse H */
  double G0_11 = dot3(a0, a0), G0_12 = dot3(a0, b0), G0_22 = dot3(b0, b0);
  double detG0 = G0_11 * G0_22 - G0_12 * G0_12;
  double H11 = G0_22 / detG0, H12 = -G0_12 / detG0, H22 = G0_11 / detG0;
  /* current metric G */
  double G11 = dot3(a, a), G12 = dot3(a, b), G22 = dot3(b, b);
  double detG = G11 * G22 - G12 * G12;
  double A0 = 0.5 * sqrt(detG0);
  double I1 = H11 * G11 + 2.0 * H12 * G12 + H22 * G22 - 2.0;
  double L = log(detG / detG0); /* log(I2 + 1) */
  double E = A0 * (0.5 * (alpha[0] - alpha[2]) * L + 0.125 * (alpha[0] + alpha[1]) * L * L +
                   alpha[2] * (0.5 * (I1 + 2.0) - 1.0));
  /* dE/dI1 and dE/dL */
  double dE_dI1 = A0 * 0.5 * alpha[2];
  double dE_dL = A0 * (0.5 * (alpha[0] - alpha[2]) + 0.25 * (alpha[0] + alpha[1]) * L);
  /* dI1/da = 2 (H11 a + H12 b), dI1/db = 2 (H12 a + H22 b)
     dL/da = (2 a G22 - 2 G12 b)/detG, dL/db = (2 b G11 - 2 G12 a)/detG */
  for (int k = 0; k < 3; k++) {
    double dI1_da = 2.0 * (H11 * a[k] + H12 * b[k]);
    double dI1_db = 2.0 * (H12 * a[k] + H22 * b[k]);
    double dL_da = (2.0 * a[k] * G22 - 2.0 * G12 * b[k]) / detG;
    double dL_db = (2.0 * b[k] * G11 - 2.0 * G12 * a[k]) / detG;
    double dE_da = dE_dI1 * dI1_da + dE_dL * dL_da;
    double dE_db = dE_dI1 * dI1_db + dE_dL * dL_db;
    g1[k] = dE_da;
    g2[k] = dE_db;
    g0[k] = -(dE_da + dE_db);
  }
  return E;
}

/* Signed volume of the tetrahedron (c, x0, x1, x2): the face's share of V in Eq. 18. */
static double face_volume(const double *x0, const double *x1, const double *x2, const double *c,
                          double *d0, double *d1, double *d2) {
  double r0[3], r1[3], r2[3], t[3];
  for (int k = 0; k < 3; k++) {
    r0[k] = x0[k] - c[k];
    r1[k] = x1[k] - c[k];
    r2[k] = x2[k] - c[k];
  }
  cross3(r1, r2, t);
  double v = dot3(r0, t) / 6.0;
  if (d0) {
    cross3(r1, r2, d0);
    cross3(r2, r0, d1);
    cross3(r0, r1, d2);
    for (int k = 0; k < 3; k++) { d0[k] /= 6.0; d1[k] /= 6.0; d2[k] /= 6.0; }
  }
  return v;
}

/* Eq. 19 for one wall plane: force on a face centroid at height gz, and its potential
   4 eps [(xi/d)^12 - (xi/d)^6] (whose negative gradient Eq. 19 is). */
static double lj_wall(double gz, double zw, double eps, double xi, double *fz) {
  double dz = gz - zw; /* R6: from the wall foot point to the centroid */
  double d = fabs(dz);
  double s6 = pow(xi / d, 6.0), s12 = s6 * s6;
  *fz = 48.0 * eps * (s12 - 0.5 * s6) * dz / (d * d);
  return 4.0 * eps * (s12 - s6);
}

/* Total nodal force, Eq. 16: phi = phi^S (Eq. 17) + phi^V (Eq. 18) + phi^W (Eq. 19).
   energies_out = {E_S, E_V, E_W}; V_out = current volume. */
void iblbref_mesh_forces(int nv, int nf, const double *q, const int32_t *faces, const double *Xref,
                         const double *centre, double V0, const double *alpha, double kV, double eps,
                         double xi, int wall_on, int volume_on, int has_walls, double z_bottom,
                         double z_top, double *phi, double *energies_out, double *V_out) {
  for (int i = 0; i < 3 * nv; i++) phi[i] = 0.0;
  double ES = 0.0, EW = 0.0, V = 0.0;
  /* strain energy and the volume sum */
  for (int j = 0; j < nf; j++) {
    int i0 = faces[3 * j], i1 = faces[3 * j + 1], i2 = faces[3 * j + 2];
    double g0[3], g1[3], g2[3];
    ES += face_strain_energy(q + 3 * i0, q + 3 * i1, q + 3 * i2, Xref + 3 * i0, Xref + 3 * i1,
                             Xref + 3 * i2, alpha, g0, g1, g2);
    for (int k = 0; k < 3; k++) {
      phi[3 * i0 + k] -= g0[k];
      phi[3 * i1 + k] -= g1[k];
      phi[3 * i2 + k] -= g2[k];
    }
    V += face_volume(q + 3 * i0, q + 3 * i1, q + 3 * i2, centre, NULL, NULL, NULL);
  }
  /* volume penalty w_V = kV (V - V0)^2 / (2 V0) */
  double EV = 0.0;
  if (volume_on) {
    EV = kV * (V - V0) * (V - V0) / (2.0 * V0);
    double coef = kV * (V - V0) / V0;
    for (int j = 0; j < nf; j++) {
      int i0 = faces[3 * j], i1 = faces[3 * j + 1], i2 = faces[3 * j + 2];
      double d0[3], d1[3], d2[3];
      face_volume(q + 3 * i0, q + 3 * i1, q + 3 * i2, centre, d0, d1, d2);
      for (int k = 0; k < 3; k++) {
        phi[3 * i0 + k] -= coef * d0[k];
        phi[3 * i1 + k] -= coef * d1[k];
        phi[3 * i2 + k] -= coef * d2[k];
      }
    }
  }
  /* wall-particle Lennard-Jones, once per face at its centroid, thirds to the vertices */
  if (wall_on && has_walls) {
    for (int j = 0; j < nf; j++) {
      int i0 = faces[3 * j], i1 = faces[3 * j + 1], i2 = faces[3 * j + 2];
      double gz = (q[3 * i0 + 2] + q[3 * i1 + 2] + q[3 * i2 + 2]) / 3.0;
      double fb, ft;
      EW += lj_wall(gz, z_bottom, eps, xi, &fb);
      EW += lj_wall(gz, z_top, eps, xi, &ft);
      double fz = fb + ft;
      phi[3 * i0 + 2] += fz / 3.0;
      phi[3 * i1 + 2] += fz / 3.0;
      phi[3 * i2 + 2] += fz / 3.0;
    }
  }
  if (energies_out) {
    energies_out[0] = ES;
    energies_out[1] = EV;
    energies_out[2] = EW;
  }
  if (V_out) *V_out = V;
}

/* Polyhedral volume of a closed, outward-oriented mesh about a fixed point c. */
double iblbref_mesh_volume(int nf, const double *q, const int32_t *faces, const double *c) {
  double V = 0.0;
  for (int j = 0; j < nf; j++)
    V += face_volume(q + 3 * faces[3 * j], q + 3 * faces[3 * j + 1], q + 3 * faces[3 * j + 2], c,
                     NULL, NULL, NULL);
  return V;
}

/* ------------------------------------------------------------------------------------ */
/* Immersed-boundary coupling, Eqs. 11-15.                                              */
/* ------------------------------------------------------------------------------------ */

/* Node classification along z (R7): 0 fluid, 1 bottom wall, 2 top wall, -1 outside. */
static int z_kind(int z, int nz, int has_walls) {
  if (!has_walls) return 0;
  if (z < 0 || z >= nz) return -1;
  if (z == 0) return 1;
  if (z == nz - 1) return 2;
  return 0;
}

/* Eq. 13 with the delta function of Eq. 14: F(x) += sum_i phi_i delta_D(x - q_i).
   F is [nz][ny][nx][3] and is accumulated into (not cleared). */
void iblbref_spread(int nx, int ny, int nz, int has_walls, int nv, const double *q,
                    const double *phi, double *F) {
  for (int v = 0; v < nv; v++) {
    const double *p = q + 3 * v;
    int base[3];
    for (int k = 0; k < 3; k++) base[k] = (int)floor(p[k]) - 1;
    for (int dz = 0; dz < 4; dz++) {
      int z = base[2] + dz;
      double wz = iblbref_phi4((double)z - p[2]);
      int kind = z_kind(z, nz, has_walls);
      if (kind != 0) continue; /* wall layer: force dropped; outside: skipped */
      int zz = wrap(z, nz);
      for (int dy = 0; dy < 4; dy++) {
        int y = base[1] + dy;
        double wy = iblbref_phi4((double)y - p[1]);
        for (int dx = 0; dx < 4; dx++) {
          int x = base[0] + dx;
          double wx = iblbref_phi4((double)x - p[0]);
          double w = wx * wy * wz;
          size_t n = ((size_t)zz * ny + wrap(y, ny)) * nx + wrap(x, nx);
          for (int k = 0; k < 3; k++) F[3 * n + k] += phi[3 * v + k] * w;
        }
      }
    }
  }
}

/* Eq. 11: qdot_i = sum_x u(x) delta_D(x - q_i). u is [nz][ny][nx][3]; wall-layer nodes use
   the wall velocity (R7). */
void iblbref_interpolate(int nx, int ny, int nz, int has_walls, const double *u_bottom,
                         const double *u_top, const double *u, int nv, const double *q,
                         double *qdot) {
  for (int v = 0; v < nv; v++) {
    const double *p = q + 3 * v;
    int base[3];
    for (int k = 0; k < 3; k++) base[k] = (int)floor(p[k]) - 1;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int dz = 0; dz < 4; dz++) {
      int z = base[2] + dz;
      double wz = iblbref_phi4((double)z - p[2]);
      int kind = z_kind(z, nz, has_walls);
      if (kind < 0) continue;
      int zz = wrap(z, nz);
      for (int dy = 0; dy < 4; dy++) {
        int y = base[1] + dy;
        double wy = iblbref_phi4((double)y - p[1]);
        for (int dx = 0; dx < 4; dx++) {
          int x = base[0] + dx;
          double wx = iblbref_phi4((double)x - p[0]);
          double w = wx * wy * wz;
          const double *un;
          if (kind == 1) un = u_bottom;
          else if (kind == 2) un = u_top;
          else un = u + 3 * (((size_t)zz * ny + wrap(y, ny)) * nx + wrap(x, nx));
          for (int k = 0; k < 3; k++) acc[k] += un[k] * w;
        }
      }
    }
    for (int k = 0; k < 3; k++) qdot[3 * v + k] = acc[k];
  }
}

/* ------------------------------------------------------------------------------------ */
/* The coupled simulation: Sec. III step order.                                        */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int nx, ny, nz, has_walls;
  double tau, rho0;
  double u_bottom[3], u_top[3], g[3];
  size_t ncell;
  double *f, *fpost; /* [19][nz][ny][nx]: populations after streaming, and after collision */
  double *F;         /* [nz][ny][nx][3]: interface force density of the last spread */
  double *u;         /* [nz][ny][nx][3]: velocity of the last step's interpolation */
  /* interface */
  int nv, nf;
  double *q, *Xref, *phi, *qdot;
  int32_t *faces;
  double centre[3], V0;
  ref_iface iface;
  long steps_done;
} ref_sim;

static size_t pidx(const ref_sim *s, int i, int x, int y, int z) {
  return (((size_t)i * s->nz + z) * s->ny + y) * s->nx + x;
}

static int is_fluid_z(const ref_sim *s, int z) {
  return !s->has_walls || (z >= 1 && z <= s->nz - 2);
}

void *iblbref_create(int nx, int ny, int nz, double tau, double rho0, const double *u_bottom,
                     const double *u_top, const double *g, int z_periodic) {
  if (nx < 1 || ny < 1 || nz < (z_periodic ? 1 : 3) || !(tau > 0.5)) return NULL;
  ref_sim *s = (ref_sim *)calloc(1, sizeof(ref_sim));
  s->nx = nx; s->ny = ny; s->nz = nz;
  s->has_walls = !z_periodic;
  s->tau = tau; s->rho0 = rho0;
  for (int k = 0; k < 3; k++) {
    s->u_bottom[k] = u_bottom[k];
    s->u_top[k] = u_top[k];
    s->g[k] = g[k];
  }
  s->ncell = (size_t)nx * ny * nz;
  s->f = (double *)calloc(Q * s->ncell, sizeof(double));
  s->fpost = (double *)calloc(Q * s->ncell, sizeof(double));
  s->F = (double *)calloc(3 * s->ncell, sizeof(double));
  s->u = (double *)calloc(3 * s->ncell, sizeof(double));
  /* initial state f = f^eq(rho0, 0) on the fluid nodes */
  double zero[3] = {0.0, 0.0, 0.0}, feq[Q];
  iblbref_equilibrium(rho0, zero, feq);
  for (int z = 0; z < nz; z++)
    if (is_fluid_z(s, z))
      for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++)
          for (int i = 0; i < Q; i++) s->f[pidx(s, i, x, y, z)] = feq[i];
  s->iface.kV = 1.0;
  s->iface.xi = 0.5;
  s->iface.volume_on = 1;
  return s;
}

void iblbref_destroy(void *h) {
  ref_sim *s = (ref_sim *)h;
  if (!s) return;
  free(s->f); free(s->fpost); free(s->F); free(s->u);
  free(s->q); free(s->Xref); free(s->phi); free(s->qdot); free(s->faces);
  free(s);
}

/* Set every fluid node to f^eq(rho, u) of the given fields ([nz][ny][nx] and [..][3]). */
void iblbref_init_equilibrium(void *h, const double *rho, const double *u) {
  ref_sim *s = (ref_sim *)h;
  for (int z = 0; z < s->nz; z++) {
    if (!is_fluid_z(s, z)) continue;
    for (int y = 0; y < s->ny; y++)
      for (int x = 0; x < s->nx; x++) {
        size_t n = ((size_t)z * s->ny + y) * s->nx + x;
        double feq[Q];
        iblbref_equilibrium(rho[n], u + 3 * n, feq);
        for (int i = 0; i < Q; i++) s->f[pidx(s, i, x, y, z)] = feq[i];
      }
  }
}

int iblbref_add_mesh(void *h, const double *verts, int nv, const int32_t *faces, int nf) {
  ref_sim *s = (ref_sim *)h;
  if (s->q || nv < 3 || nf < 1) return -1;
  s->nv = nv; s->nf = nf;
  s->q = (double *)malloc(sizeof(double) * 3 * nv);
  s->Xref = (double *)malloc(sizeof(double) * 3 * nv);
  s->phi = (double *)calloc(3 * nv, sizeof(double));
  s->qdot = (double *)calloc(3 * nv, sizeof(double));
  s->faces = (int32_t *)malloc(sizeof(int32_t) * 3 * nf);
  memcpy(s->q, verts, sizeof(double) * 3 * nv);
  memcpy(s->Xref, verts, sizeof(double) * 3 * nv);
  memcpy(s->faces, faces, sizeof(int32_t) * 3 * nf);
  s->centre[0] = s->centre[1] = s->centre[2] = 0.0;
  for (int v = 0; v < nv; v++)
    for (int k = 0; k < 3; k++) s->centre[k] += verts[3 * v + k] / nv;
  s->V0 = iblbref_mesh_volume(nf, s->q, s->faces, s->centre);
  return 0;
}

/* Replace the current vertex positions; the reference shape stays the one added. */
void iblbref_set_vertices(void *h, const double *q) {
  ref_sim *s = (ref_sim *)h;
  memcpy(s->q, q, sizeof(double) * 3 * s->nv);
}

void iblbref_set_interface(void *h, const double *alpha, double kV, double eps, double xi,
                           int wall_on, int volume_on) {
  ref_sim *s = (ref_sim *)h;
  for (int k = 0; k < 3; k++) s->iface.alpha[k] = alpha[k];
  s->iface.kV = kV;
  s->iface.eps = eps;
  s->iface.xi = xi;
  s->iface.wall_on = wall_on;
  s->iface.volume_on = volume_on;
}

static void compute_forces(ref_sim *s, double *energies, double *V) {
  iblbref_mesh_forces(s->nv, s->nf, s->q, s->faces, s->Xref, s->centre, s->V0, s->iface.alpha,
                      s->iface.kV, s->iface.eps, s->iface.xi, s->iface.wall_on,
                      s->iface.volume_on, s->has_walls, 0.5, s->nz - 1.5, s->phi, energies, V);
}

/* One step in the order of Sec. III. */
static void sim_step(ref_sim *s) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  /* interface forces, Eq. 16, then spreading, Eq. 13 */
  memset(s->F, 0, sizeof(double) * 3 * s->ncell);
  if (s->q) {
    compute_forces(s, NULL, NULL);
    iblbref_spread(nx, ny, nz, s->has_walls, s->nv, s->q, s->phi, s->F);
  }
  /* collision, Eq. 9 right-hand side, with the total force F + g */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; z++) {
    if (!is_fluid_z(s, z)) continue;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = ((size_t)z * ny + y) * nx + x;
        double f[Q], fo[Q], Ft[3];
        for (int k = 0; k < 3; k++) Ft[k] = s->F[3 * n + k] + s->g[k];
        for (int i = 0; i < Q; i++) f[i] = s->f[pidx(s, i, x, y, z)];
        iblbref_collide_node(s->tau, f, Ft, fo);
        for (int i = 0; i < Q; i++) s->fpost[pidx(s, i, x, y, z)] = fo[i];
      }
  }
  /* propagation, Eq. 9 left-hand side, with half-way bounce-back at the walls (R7) */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; z++) {
    if (!is_fluid_z(s, z)) continue;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++)
        for (int i = 0; i < Q; i++) {
          double fo = s->fpost[pidx(s, i, x, y, z)];
          int zd = z + CVEL[i][2];
          int kind = z_kind(zd, nz, s->has_walls);
          if (kind == 0) {
            s->f[pidx(s, i, wrap(x + CVEL[i][0], nx), wrap(y + CVEL[i][1], ny), wrap(zd, nz))] = fo;
          } else {
            const double *uw = (kind == 1) ? s->u_bottom : s->u_top;
            double c[3] = {CVEL[i][0], CVEL[i][1], CVEL[i][2]};
            s->f[pidx(s, opposite(i), x, y, z)] = fo - 2.0 * weight(i) * s->rho0 * dot3(c, uw) * INV_CS2;
          }
        }
  }
  /* fluid velocity from the streamed populations with the same force (R8) */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t n = ((size_t)z * ny + y) * nx + x;
        if (!is_fluid_z(s, z)) {
          const double *uw = (z == 0) ? s->u_bottom : s->u_top;
          for (int k = 0; k < 3; k++) s->u[3 * n + k] = uw[k];
          continue;
        }
        double f[Q], Ft[3], rho;
        for (int k = 0; k < 3; k++) Ft[k] = s->F[3 * n + k] + s->g[k];
        for (int i = 0; i < Q; i++) f[i] = s->f[pidx(s, i, x, y, z)];
        iblbref_moments(f, Ft, &rho, s->u + 3 * n);
      }
  /* interpolation, Eq. 11, and the Euler update, Eq. 12 */
  if (s->q) {
    iblbref_interpolate(nx, ny, nz, s->has_walls, s->u_bottom, s->u_top, s->u, s->nv, s->q,
                        s->qdot);
    for (int i = 0; i < 3 * s->nv; i++) s->q[i] += s->qdot[i];
  }
  s->steps_done++;
}

void iblbref_step(void *h, int nsteps) {
  for (int t = 0; t < nsteps; t++) sim_step((ref_sim *)h);
}

/* rho [nz][ny][nx] and u [nz][ny][nx][3] of the current (post-streaming) state; u carries
   the half force of the last spread field (zero before the first step). Wall nodes report
   rho0 and the wall velocity. */
void iblbref_read_fields(void *h, double *rho, double *u) {
  ref_sim *s = (ref_sim *)h;
  for (int z = 0; z < s->nz; z++)
    for (int y = 0; y < s->ny; y++)
      for (int x = 0; x < s->nx; x++) {
        size_t n = ((size_t)z * s->ny + y) * s->nx + x;
        if (!is_fluid_z(s, z)) {
          const double *uw = (z == 0) ? s->u_bottom : s->u_top;
          rho[n] = s->rho0;
          for (int k = 0; k < 3; k++) u[3 * n + k] = uw[k];
          continue;
        }
        double f[Q], Ft[3];
        for (int k = 0; k < 3; k++) Ft[k] = s->F[3 * n + k] + s->g[k];
        for (int i = 0; i < Q; i++) f[i] = s->f[pidx(s, i, x, y, z)];
        iblbref_moments(f, Ft, rho + n, u + 3 * n);
      }
}

/* Populations [19][nz][ny][nx] after the last streaming. */
void iblbref_read_populations(void *h, double *f) {
  ref_sim *s = (ref_sim *)h;
  memcpy(f, s->f, sizeof(double) * Q * s->ncell);
}

/* Replace the populations [19][nz][ny][nx] (the post-streaming state the next step reads). */
void iblbref_set_populations(void *h, const double *f) {
  ref_sim *s = (ref_sim *)h;
  memcpy(s->f, f, sizeof(double) * Q * s->ncell);
}

/* Threads of the per-node loops (see the header); returns the count in effect, 1 without
   OpenMP. n <= 0 keeps the current setting. */
int iblbref_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

void iblbref_read_vertices(void *h, double *q) {
  ref_sim *s = (ref_sim *)h;
  memcpy(q, s->q, sizeof(double) * 3 * s->nv);
}

void iblbref_read_vertex_velocities(void *h, double *qdot) {
  ref_sim *s = (ref_sim *)h;
  memcpy(qdot, s->qdot, sizeof(double) * 3 * s->nv);
}

/* Nodal forces at the current vertex positions (computed now), energies {E_S, E_V, E_W}. */
void iblbref_read_forces(void *h, double *phi, double *energies) {
  ref_sim *s = (ref_sim *)h;
  compute_forces(s, energies, NULL);
  memcpy(phi, s->phi, sizeof(double) * 3 * s->nv);
}

/* Force density [nz][ny][nx][3] spread from the forces at the current vertex positions. */
void iblbref_read_force_field(void *h, double *F) {
  ref_sim *s = (ref_sim *)h;
  memset(F, 0, sizeof(double) * 3 * s->ncell);
  compute_forces(s, NULL, NULL);
  iblbref_spread(s->nx, s->ny, s->nz, s->has_walls, s->nv, s->q, s->phi, F);
}

void iblbref_read_volume(void *h, double *V, double *V0) {
  ref_sim *s = (ref_sim *)h;
  *V = iblbref_mesh_volume(s->nf, s->q, s->faces, s->centre);
  *V0 = s->V0;
}

long iblbref_steps_done(void *h) { return ((ref_sim *)h)->steps_done; }
