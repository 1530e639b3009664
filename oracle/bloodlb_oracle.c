/*
 * bloodlb_oracle.c -- plain, slow FP64 restatement of the coupled time step of
 * Janoschek, Toschi & Harting, "A simplified particulate model for
 * coarse-grained hemodynamics simulations" (arXiv:1005.2594).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product path never does.  It shares
 * no code, header, table or helper with the CUDA path.
 *
 * Every step is written out in the order of the method, in double precision,
 * with no blocking, fusion or reordering.  Compile with -ffp-contract=off so
 * that the inside test of the re-discretisation is evaluated with exactly the
 * rounding written here.
 *
 * Method, by section of the paper:
 *   Sec. II, Eq. (col),(adv)   BGK collision then advection
 *   Sec. II, Eq. (neq)         equilibrium to third order in u, c_s^2 = 1/3,
 *                              weights 1/3, 1/18, 1/36
 *   Sec. II, Eq. (lbe-bb),(c),(lbe-bb-corr)
 *                              mid-link bounce-back with moving-wall term C
 *   Sec. II, Eq. (deltap)      momentum exchange (2 n_rbar + C) c_rbar per link
 *   Sec. II (fill/drain)       covered nodes lose their fluid, freed nodes get
 *                              n^eq(rho_bar, u_rigid); momentum goes to the cell
 *   Sec. II, Eq. (deltapppp),(deltapppm)
 *                              particle-particle / particle-wall contact links
 *   Sec. II (single occupancy) first-arrival owner rule
 *   Sec. III, Eq. (phi),(epsilon),(sigma),(sigmaw)
 *                              Berne-Pechukas-scaled Hookean potentials
 *   Sec. II (leap-frog on unit quaternions)
 *   Sec. IV (Lees-Edwards shear across the x plane, reflective cell
 *                              boundary, momentum transfer Delta p_LE of Eq. mu)
 *
 * Where the paper is silent the readings are (numbered as in the design notes):
 *   Q1 body force: Guo forcing, u = (j + rho g / 2) / rho
 *   Q2 v_b at the link midpoint, rho(y,t) local in C
 *   Q3 C uses V, Omega of t+1/2, solved jointly with the link forces
 *      (implicit coupling); fill uses V, Omega of t+1/2 and X(t+1)
 *   Q4 lab-frame angular-momentum leap-frog, exact quaternion exponential
 *   Q5 simultaneous arrival: lowest particle index; s == 1 counts as inside
 *   Q6 owner change p->q: uncover by p, then cover by q
 *   Q7 n_rbar in Eq. (deltap) is the post-collision population
 *   Q8 neutrally buoyant solid ellipsoid, analytic mass and inertia
 *   Q9 epsilon may carry the Gay-Berne factor eps2^mu (paper: mu = 0, nu = 1)
 *   Q10 a walled axis has solid layers at index 0 and N-1
 *   Q25 Lees-Edwards: offset D = U t, linear interpolation along z, the
 *       equilibrium part of a crossing population moved by -+U with its
 *       source's rho and u; Delta p_LE the mean flux of the two frames; cells
 *       reflected after the step's coupling, before they move
 *
 * Direction numbering (the interface order, also used by the link lists):
 *   0 (0,0,0); 1..6 (+x,-x,+y,-y,+z,-z); 7..18 the twelve (+-1,+-1,0)-type
 *   vectors, each followed by its opposite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19
#define FLUID (-1)
/* a wall node with wall id w (0..7) stores owner = -2 - w */
#define IS_WALL(o) ((o) <= -2)
#define WALL_ID(o) (-2 - (o))
#define NWALL 8

static const int CX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

/* Sec. II: alpha = 1/3 (rest), 1/18 (|c| = 1), 1/36 (|c| = sqrt 2) */
static double weight(int r) {
  int c2 = CX[r] * CX[r] + CY[r] * CY[r] + CZ[r] * CZ[r];
  if (c2 == 0) return 1.0 / 3.0;
  if (c2 == 1) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

/* index of the direction with c = -c_r, found by search (no table) */
static int opposite(int r) {
  for (int s = 0; s < NQ; ++s)
    if (CX[s] == -CX[r] && CY[s] == -CY[r] && CZ[s] == -CZ[r]) return s;
  return -1;
}

typedef struct {
  int nx, ny, nz;
  int periodic[3];
  double wall_vel[NWALL][3];
  double tau, rho0;
  double g[3];
  int body_force_on_cells;
  /* cells */
  double R_par, R_perp;
  double sig_par, sig_perp;
  double eps, eps_w, sig_w;
  double mu, nu, chi_prime;
  double r_cut;
  double rho_p;
  int move_particles; /* 0 held fixed, 1 free (implicit coupling), 2 prescribed V, Omega */
} orc_params;

typedef struct {
  orc_params p;
  long N;
  double *n;     /* N x 19: populations n_r(x,t) before collision */
  double *nstar; /* N x 19: post-collision populations of the current step */
  double *nnew;  /* N x 19: populations of t+1 */
  double *rho;   /* N: local density of the current step */
  int32_t *owner;
  int np;
  double *X, *q, *V, *L, *Om; /* state: X(t), q(t), V(t-1/2), L(t-1/2), Omega(t-1/2) */
  double *Fh, *Th;            /* link forces of the last step: bounce-back + contact */
  double *Fc, *Tc;            /* contact-link part only (diagnostic) */
  double *Fp, *Tp;            /* pair + wall potential forces of the last step */
  double *Fw, *Tw;            /* wall part of Fp, Tp alone (diagnostic) */
  double *PF, *PT;            /* fill/drain impulses waiting for the next integration */
  double *Ftot, *Ttot;        /* total force / torque used in the last integration */
  double wallmom[NWALL][3];   /* momentum given to each wall by its links in the last step */
  /* bookkeeping of the last step */
  double sumC, mass_created, mass_deleted;
  long n_covered, n_uncovered, n_switched;
  long t;
  double *u; /* N x 3: velocity of the current step's collision */
  /* Lees-Edwards shear across the plane between x = nx-1 and x = 0 (Sec. IV,
     reading Q25): the image above (x + nx) is displaced by D = U le_t along z
     and moves with velocity offset U along z; cells reflect within le_dr of
     the plane */
  int le_on;
  double le_U, le_dr;
  long le_t;
  double le_P, le_Psum;   /* z-momentum moved across the plane along +x: last step, summed */
  long le_n, le_reflect;  /* steps summed, cell reflections so far */
  long le_bad;            /* crossings whose source was not fluid (the planes must stay fluid) */
} orc_state;

/* ------------------------------------------------------------------ */
/* lattice helpers                                                     */

static long node_index(const orc_params *p, int x, int y, int z) {
  return (long)x + (long)p->nx * ((long)y + (long)p->ny * (long)z);
}

static int wrap(int v, int n) {
  if (v < 0) return v + n;
  if (v >= n) return v - n;
  return v;
}

static long neighbour(const orc_params *p, long idx, int r, int sign) {
  int x = (int)(idx % p->nx);
  int y = (int)((idx / p->nx) % p->ny);
  int z = (int)(idx / ((long)p->nx * p->ny));
  return node_index(p, wrap(x + sign * CX[r], p->nx), wrap(y + sign * CY[r], p->ny),
                    wrap(z + sign * CZ[r], p->nz));
}

static void node_coords(const orc_params *p, long idx, double xyz[3]) {
  xyz[0] = (double)(idx % p->nx);
  xyz[1] = (double)((idx / p->nx) % p->ny);
  xyz[2] = (double)(idx / ((long)p->nx * p->ny));
}

/* minimum image of a displacement along axis k (periodic axes only) */
static double min_image(const orc_params *p, int k, double d) {
  int n = k == 0 ? p->nx : (k == 1 ? p->ny : p->nz);
  if (!p->periodic[k]) return d;
  double half = 0.5 * (double)n;
  if (d > half) return d - (double)n;
  if (d < -half) return d + (double)n;
  return d;
}

static void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ------------------------------------------------------------------ */
/* Sec. II, Eq. (neq): third-order equilibrium, c_s^2 = 1/3            */

void orc_equilibrium(double rho, const double u[3], double out[NQ]) {
  const double cs2 = 1.0 / 3.0;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int r = 0; r < NQ; ++r) {
    double cu = CX[r] * u[0] + CY[r] * u[1] + CZ[r] * u[2];
    out[r] = rho * weight(r) *
             (1.0 + cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2) +
              cu * cu * cu / (6.0 * cs2 * cs2 * cs2) - uu * cu / (2.0 * cs2 * cs2));
  }
}

/* Guo source term S_r for force density Fd at velocity u (reading Q1) */
static void guo_source(const double u[3], const double Fd[3], double out[NQ]) {
  const double cs2 = 1.0 / 3.0;
  for (int r = 0; r < NQ; ++r) {
    double c[3] = {CX[r], CY[r], CZ[r]};
    double cu = dot3(c, u);
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += ((c[k] - u[k]) / cs2 + cu * c[k] / (cs2 * cs2)) * Fd[k];
    out[r] = weight(r) * s;
  }
}

/* ------------------------------------------------------------------ */
/* particle geometry                                                   */

/* symmetry axis o = R(q) e_z, q = (w,x,y,z).  The expression is evaluated
   exactly as written; the inside test below depends on its rounding. */
void orc_axis(const double q[4], double o[3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  o[0] = 2.0 * (x * z + w * y);
  o[1] = 2.0 * (y * z - w * x);
  o[2] = 1.0 - 2.0 * (x * x + y * y);
}

/* rotation matrix of a unit quaternion (columns are body axes in the lab) */
static void rotmat(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Sec. II: node x is inside cell p when s <= 1 (reading Q5), with
   s = d_par^2 / R_par^2 + (|d|^2 - d_par^2) / R_perp^2, d = x - X (min image).
   1/R^2 are formed once by the caller. */
static int inside(const orc_params *p, const double xyz[3], const double X[3], const double o[3],
                  double inv_rpar2, double inv_rperp2) {
  double d0 = min_image(p, 0, xyz[0] - X[0]);
  double d1 = min_image(p, 1, xyz[1] - X[1]);
  double d2 = min_image(p, 2, xyz[2] - X[2]);
  double dpar = d0 * o[0] + d1 * o[1] + d2 * o[2];
  double dd = d0 * d0 + d1 * d1 + d2 * d2;
  double s = dpar * dpar * inv_rpar2 + (dd - dpar * dpar) * inv_rperp2;
  return s <= 1.0;
}

static double cell_mass(const orc_params *p) {
  return p->rho_p * (4.0 / 3.0) * M_PI * p->R_perp * p->R_perp * p->R_par;
}

/* Omega = I_lab^-1 L with I_lab = R diag(I_perp, I_perp, I_par) R^T (reading Q4/Q8) */
static void omega_from_L(const orc_params *p, const double q[4], const double L[3], double Om[3]) {
  double m = cell_mass(p);
  double Iperp = m * (p->R_par * p->R_par + p->R_perp * p->R_perp) / 5.0;
  double Ipar = 2.0 * m * p->R_perp * p->R_perp / 5.0;
  double R[3][3];
  rotmat(q, R);
  double Lb[3]; /* body frame: R^T L */
  for (int i = 0; i < 3; ++i) Lb[i] = R[0][i] * L[0] + R[1][i] * L[1] + R[2][i] * L[2];
  double wb[3] = {Lb[0] / Iperp, Lb[1] / Iperp, Lb[2] / Ipar};
  for (int i = 0; i < 3; ++i) Om[i] = R[i][0] * wb[0] + R[i][1] * wb[1] + R[i][2] * wb[2];
}

/* ------------------------------------------------------------------ */
/* Sec. III potentials                                                 */

/* Cell-cell pair, Eq. (phi),(epsilon),(sigma).  r = Xj - Xi (already min
   image).  With mu != 0 the strength carries the Gay-Berne factor
   eps2^mu, eps2 being the bracket of Eq. (sigma) with chi' (reading Q9).
   Returns phi; writes forces on i and j and torques on i and j. */
double orc_pair(const orc_params *p, const double rvec[3], const double oi[3], const double oj[3],
                double Fi[3], double Fj[3], double Ti[3], double Tj[3]) {
  for (int k = 0; k < 3; ++k) Fi[k] = Fj[k] = Ti[k] = Tj[k] = 0.0;
  double r = sqrt(dot3(rvec, rvec));
  if (r <= 0.0) return 0.0;
  double rh[3] = {rvec[0] / r, rvec[1] / r, rvec[2] / r};
  double sp2 = p->sig_par * p->sig_par, sq2 = p->sig_perp * p->sig_perp;
  double chi = (sp2 - sq2) / (sp2 + sq2);
  double sigbar = 2.0 * p->sig_perp;
  double a = dot3(rh, oi), b = dot3(rh, oj), c = dot3(oi, oj);
  /* Eq. (sigma): sigma = sigbar / sqrt(S) */
  double S = 1.0 - 0.5 * chi * ((a + b) * (a + b) / (1.0 + chi * c) + (a - b) * (a - b) / (1.0 - chi * c));
  double sigma = sigbar / sqrt(S);
  if (r >= sigma) return 0.0;
  /* Eq. (epsilon), general Gay-Berne exponents (paper: nu = 1, mu = 0) */
  double e1 = 1.0 - chi * chi * c * c;
  double cp = p->chi_prime;
  double e2 = 1.0 - 0.5 * cp * ((a + b) * (a + b) / (1.0 + cp * c) + (a - b) * (a - b) / (1.0 - cp * c));
  double eps = p->eps * pow(e1, -0.5 * p->nu) * (p->mu != 0.0 ? pow(e2, p->mu) : 1.0);
  /* Eq. (phi) */
  double h = 1.0 - r / sigma;
  double phi = eps * h * h;
  /* partial derivatives of S, eps2 with respect to a, b, c */
  double dSa = -chi * ((a + b) / (1.0 + chi * c) + (a - b) / (1.0 - chi * c));
  double dSb = -chi * ((a + b) / (1.0 + chi * c) - (a - b) / (1.0 - chi * c));
  double dSc = 0.5 * chi * chi *
               ((a + b) * (a + b) / ((1.0 + chi * c) * (1.0 + chi * c)) -
                (a - b) * (a - b) / ((1.0 - chi * c) * (1.0 - chi * c)));
  double de2a = -cp * ((a + b) / (1.0 + cp * c) + (a - b) / (1.0 - cp * c));
  double de2b = -cp * ((a + b) / (1.0 + cp * c) - (a - b) / (1.0 - cp * c));
  double de2c = 0.5 * cp * cp *
                ((a + b) * (a + b) / ((1.0 + cp * c) * (1.0 + cp * c)) -
                 (a - b) * (a - b) / ((1.0 - cp * c) * (1.0 - cp * c)));
  double mu = p->mu;
  double eps_a = mu != 0.0 ? eps * mu * de2a / e2 : 0.0;
  double eps_b = mu != 0.0 ? eps * mu * de2b / e2 : 0.0;
  double eps_c = eps * (p->nu * chi * chi * c / e1 + (mu != 0.0 ? mu * de2c / e2 : 0.0));
  /* phi(r, a, b, c): d phi = h^2 d eps + 2 eps h (r / sigma^2) d sigma - 2 eps h / sigma d r,
     d sigma = -sigma / (2 S) dS */
  double k = eps * h * r / (sigma * S);
  double phi_r = -2.0 * eps * h / sigma;
  double phi_a = h * h * eps_a - k * dSa;
  double phi_b = h * h * eps_b - k * dSb;
  double phi_c = h * h * eps_c - k * dSc;
  /* d phi / d rvec, with da/drvec = (oi - a rh) / r, db/drvec = (oj - b rh) / r */
  double g[3];
  for (int m = 0; m < 3; ++m)
    g[m] = phi_r * rh[m] + phi_a * (oi[m] - a * rh[m]) / r + phi_b * (oj[m] - b * rh[m]) / r;
  for (int m = 0; m < 3; ++m) {
    Fi[m] = g[m];  /* rvec = Xj - Xi: F_i = -d phi / d X_i = + d phi / d rvec */
    Fj[m] = -g[m];
  }
  /* torques tau = -o x d phi / d o, o treated as a free vector */
  double dpi[3], dpj[3];
  for (int m = 0; m < 3; ++m) {
    dpi[m] = phi_a * rh[m] + phi_c * oj[m];
    dpj[m] = phi_b * rh[m] + phi_c * oi[m];
  }
  cross(oi, dpi, Ti);
  cross(oj, dpj, Tj);
  for (int m = 0; m < 3; ++m) {
    Ti[m] = -Ti[m];
    Tj[m] = -Tj[m];
  }
  return phi;
}

/* Cell-wall, Eq. (phi) with Eq. (sigmaw) and fixed strength eps_w.
   r = x_wall - X_i (already min image).  Returns phi; force and torque on i. */
double orc_wall(const orc_params *p, const double rvec[3], const double oi[3], double Fi[3], double Ti[3]) {
  for (int k = 0; k < 3; ++k) Fi[k] = Ti[k] = 0.0;
  double r = sqrt(dot3(rvec, rvec));
  if (r <= 0.0) return 0.0;
  double rh[3] = {rvec[0] / r, rvec[1] / r, rvec[2] / r};
  double sp2 = p->sig_par * p->sig_par, sq2 = p->sig_perp * p->sig_perp, sw2 = p->sig_w * p->sig_w;
  double sigbar_w = sqrt(sq2 + sw2);
  double chi_w = (sp2 - sq2) / (sp2 + sw2);
  double a = dot3(rh, oi);
  double D = 1.0 - chi_w * a * a;
  double sigma = sigbar_w / sqrt(D);
  if (r >= sigma) return 0.0;
  double eps = p->eps_w;
  double h = 1.0 - r / sigma;
  double phi = eps * h * h;
  double dsig_a = sigma * chi_w * a / D;
  double phi_r = -2.0 * eps * h / sigma;
  double phi_a = 2.0 * eps * h * r / (sigma * sigma) * dsig_a;
  double g[3];
  for (int m = 0; m < 3; ++m) g[m] = phi_r * rh[m] + phi_a * (oi[m] - a * rh[m]) / r;
  for (int m = 0; m < 3; ++m) Fi[m] = g[m];
  double dpo[3] = {phi_a * rh[0], phi_a * rh[1], phi_a * rh[2]};
  cross(oi, dpo, Ti);
  for (int m = 0; m < 3; ++m) Ti[m] = -Ti[m];
  return phi;
}

/* ------------------------------------------------------------------ */
/* Sec. II rigid-body leap-frog on unit quaternions (reading Q4):
     V(t+1/2) = V(t-1/2) + F / m,     X(t+1) = X(t) + V(t+1/2), wrapped,
     L(t+1/2) = L(t-1/2) + T,         Omega = I_lab(q(t))^-1 L(t+1/2),
     q(t+1) = normalize(exp(Omega / 2) (x) q(t)), the exact rotation by
     |Omega| about Omega / |Omega| applied in the lab frame.              */

/* X += V (wrapped on periodic axes); q <- exp(Om / 2) (x) q, normalised */
static void rigid_advance(const orc_params *p, double X[3], double q[4], const double V[3], const double Om[3]) {
  int n[3] = {p->nx, p->ny, p->nz};
  for (int k = 0; k < 3; ++k) {
    X[k] += V[k];
    if (p->periodic[k]) {
      if (X[k] < 0.0) X[k] += (double)n[k];
      else if (X[k] >= (double)n[k]) X[k] -= (double)n[k];
    }
  }
  double th = sqrt(dot3(Om, Om));
  double dq[4] = {1.0, 0.0, 0.0, 0.0};
  if (th > 0.0) {
    double sh = sin(0.5 * th) / th;
    dq[0] = cos(0.5 * th); dq[1] = Om[0] * sh; dq[2] = Om[1] * sh; dq[3] = Om[2] * sh;
  }
  double nq[4];
  nq[0] = dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3];
  nq[1] = dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2];
  nq[2] = dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1];
  nq[3] = dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0];
  double nn = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2] + nq[3] * nq[3]);
  for (int k = 0; k < 4; ++k) q[k] = nq[k] / nn;
}

/* free rigid-body step with a given force and torque */
void orc_integrate_one(const orc_params *p, double X[3], double q[4], double V[3], double L[3], double Om[3],
                       const double F[3], const double T[3]) {
  double m = cell_mass(p);
  for (int k = 0; k < 3; ++k) {
    V[k] += F[k] / m;
    L[k] += T[k];
  }
  omega_from_L(p, q, L, Om);
  rigid_advance(p, X, q, V, Om);
}

/* lab-frame inertia tensor R diag(I_perp, I_perp, I_par) R^T */
static void inertia_lab(const orc_params *p, const double q[4], double I[3][3]) {
  double m = cell_mass(p);
  double Iperp = m * (p->R_par * p->R_par + p->R_perp * p->R_perp) / 5.0;
  double Ipar = 2.0 * m * p->R_perp * p->R_perp / 5.0;
  double R[3][3];
  rotmat(q, R);
  double d[3] = {Iperp, Iperp, Ipar};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
      for (int k = 0; k < 3; ++k) v += R[i][k] * d[k] * R[j][k];
      I[i][j] = v;
    }
}

/* Gaussian elimination with partial pivoting: A x = b for n <= 6 */
static void solve_dense(int n, double A[6][6], double b[6], double x[6]) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
      double t = b[c]; b[c] = b[piv]; b[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r][c] / A[c][c];
      for (int k = c; k < n; ++k) A[r][k] -= f * A[c][k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double v = b[r];
    for (int k = r + 1; k < n; ++k) v -= A[r][k] * x[k];
    x[r] = v / A[r][r];
  }
}

/* ------------------------------------------------------------------ */
/* state                                                               */

static void *xcalloc(long n, long sz) {
  void *v = calloc((size_t)(n > 0 ? n : 1), (size_t)sz);
  return v;
}

static void free_particles(orc_state *s) {
  double **arrs[] = {&s->X, &s->q, &s->V, &s->L, &s->Om, &s->Fh, &s->Th, &s->Fc, &s->Tc,
                     &s->Fp, &s->Tp, &s->Fw, &s->Tw, &s->PF, &s->PT, &s->Ftot, &s->Ttot};
  for (unsigned i = 0; i < sizeof(arrs) / sizeof(arrs[0]); ++i) {
    free(*arrs[i]);
    *arrs[i] = NULL;
  }
  s->np = 0;
}

void orc_destroy(orc_state *s) {
  if (!s) return;
  free(s->n); free(s->nstar); free(s->nnew); free(s->rho); free(s->owner); free(s->u);
  free_particles(s);
  free(s);
}

/* Q10: a non-periodic axis carries solid wall layers at index 0 and N-1.
   Face walls are numbered x-,x+,y-,y+,z-,z+ = 0..5; an edge node takes the
   first face in that order. */
static int face_wall(const orc_params *p, int x, int y, int z) {
  int c[3] = {x, y, z};
  int n[3] = {p->nx, p->ny, p->nz};
  for (int k = 0; k < 3; ++k) {
    if (p->periodic[k]) continue;
    if (c[k] == 0) return 2 * k;
    if (c[k] == n[k] - 1) return 2 * k + 1;
  }
  return -1;
}

orc_state *orc_create(const orc_params *p) {
  orc_state *s = (orc_state *)xcalloc(1, sizeof(orc_state));
  s->p = *p;
  s->N = (long)p->nx * p->ny * p->nz;
  s->n = (double *)xcalloc(s->N * NQ, sizeof(double));
  s->nstar = (double *)xcalloc(s->N * NQ, sizeof(double));
  s->nnew = (double *)xcalloc(s->N * NQ, sizeof(double));
  s->rho = (double *)xcalloc(s->N, sizeof(double));
  s->u = (double *)xcalloc(3 * s->N, sizeof(double));
  s->owner = (int32_t *)xcalloc(s->N, sizeof(int32_t));
  double zero[3] = {0, 0, 0}, feq[NQ];
  orc_equilibrium(p->rho0, zero, feq); /* resting fluid at rho_bar */
  for (int z = 0; z < p->nz; ++z)
    for (int y = 0; y < p->ny; ++y)
      for (int x = 0; x < p->nx; ++x) {
        long i = node_index(p, x, y, z);
        int w = face_wall(p, x, y, z);
        s->owner[i] = w >= 0 ? -2 - w : FLUID;
        for (int r = 0; r < NQ; ++r) s->n[i * NQ + r] = s->owner[i] == FLUID ? feq[r] : 0.0;
      }
  return s;
}

/* extra static walls: mask[i] = k (1..8) makes node i a wall with id k-1 */
void orc_set_walls(orc_state *s, const uint8_t *mask) {
  for (long i = 0; i < s->N; ++i) {
    if (mask[i] == 0) continue;
    s->owner[i] = -2 - (int)(mask[i] - 1);
    for (int r = 0; r < NQ; ++r) s->n[i * NQ + r] = 0.0;
  }
}

/* ------------------------------------------------------------------ */
/* Sec. II re-discretisation with the first-arrival rule and fill/drain */

static void rediscretise(orc_state *s, int first_call) {
  orc_params *p = &s->p;
  double inv_rpar2 = 1.0 / (p->R_par * p->R_par);
  double inv_rperp2 = 1.0 / (p->R_perp * p->R_perp);
  double *o = (double *)xcalloc(3 * (long)s->np, sizeof(double));
  for (int k = 0; k < s->np; ++k) orc_axis(&s->q[4 * k], &o[3 * k]);
  int32_t *nowner = (int32_t *)xcalloc(s->N, sizeof(int32_t));
  for (long i = 0; i < s->N; ++i) {
    int32_t old = s->owner[i];
    if (IS_WALL(old)) { nowner[i] = old; continue; }
    double xyz[3];
    node_coords(p, i, xyz);
    if (!first_call && old >= 0 && inside(p, xyz, &s->X[3 * old], &o[3 * old], inv_rpar2, inv_rperp2)) {
      nowner[i] = old; /* first arrival keeps the node */
      continue;
    }
    int32_t nw = FLUID;
    for (int k = 0; k < s->np; ++k)
      if (inside(p, xyz, &s->X[3 * k], &o[3 * k], inv_rpar2, inv_rperp2)) { nw = k; break; }
    nowner[i] = nw;
  }
  free(o);
  s->mass_created = s->mass_deleted = 0.0;
  s->n_covered = s->n_uncovered = s->n_switched = 0;
  for (long i = 0; i < s->N; ++i) {
    int32_t old = s->owner[i], nw = nowner[i];
    if (old == nw) continue;
    double xyz[3];
    node_coords(p, i, xyz);
    double *ni = &s->n[i * NQ];
    /* rigid velocity of the old owner at this node, Q3: V, Omega of t+1/2, X(t+1) */
    double u_old[3] = {0, 0, 0}, arm_old[3] = {0, 0, 0};
    if (old >= 0) {
      for (int k = 0; k < 3; ++k) arm_old[k] = min_image(p, k, xyz[k] - s->X[3 * old + k]);
      double w[3];
      cross(&s->Om[3 * old], arm_old, w);
      for (int k = 0; k < 3; ++k) u_old[k] = s->V[3 * old + k] + w[k];
    }
    if (old == FLUID && nw >= 0) {
      /* covered: the fluid is deleted, its momentum goes to the new owner */
      double mom[3] = {0, 0, 0}, mass = 0.0;
      for (int r = 0; r < NQ; ++r) {
        mass += ni[r];
        mom[0] += ni[r] * CX[r]; mom[1] += ni[r] * CY[r]; mom[2] += ni[r] * CZ[r];
      }
      s->n_covered++;
      if (!first_call) {
        double arm[3], tq[3];
        for (int k = 0; k < 3; ++k) arm[k] = min_image(p, k, xyz[k] - s->X[3 * nw + k]);
        cross(arm, mom, tq);
        for (int k = 0; k < 3; ++k) { s->PF[3 * nw + k] += mom[k]; s->PT[3 * nw + k] += tq[k]; }
        s->mass_deleted += mass;
      }
      for (int r = 0; r < NQ; ++r) ni[r] = 0.0;
    } else if (old >= 0 && nw == FLUID) {
      /* uncovered: new fluid at n^eq(rho_bar, u_rigid); its momentum is taken from the old owner */
      orc_equilibrium(p->rho0, u_old, ni);
      double mass = 0.0;
      for (int r = 0; r < NQ; ++r) mass += ni[r];
      s->mass_created += mass;
      s->n_uncovered++;
      double mom[3] = {p->rho0 * u_old[0], p->rho0 * u_old[1], p->rho0 * u_old[2]}, tq[3];
      cross(arm_old, mom, tq);
      for (int k = 0; k < 3; ++k) { s->PF[3 * old + k] -= mom[k]; s->PT[3 * old + k] -= tq[k]; }
    } else if (old >= 0 && nw >= 0) {
      /* Q6: uncover by the old owner, then cover by the new one */
      s->n_switched++;
      double mom[3] = {p->rho0 * u_old[0], p->rho0 * u_old[1], p->rho0 * u_old[2]}, tq[3], arm[3];
      cross(arm_old, mom, tq);
      for (int k = 0; k < 3; ++k) { s->PF[3 * old + k] -= mom[k]; s->PT[3 * old + k] -= tq[k]; }
      for (int k = 0; k < 3; ++k) arm[k] = min_image(p, k, xyz[k] - s->X[3 * nw + k]);
      cross(arm, mom, tq);
      for (int k = 0; k < 3; ++k) { s->PF[3 * nw + k] += mom[k]; s->PT[3 * nw + k] += tq[k]; }
    }
  }
  memcpy(s->owner, nowner, sizeof(int32_t) * s->N);
  free(nowner);
}

/* Sets the particle state X(t), q(t), V(t-1/2), L(t-1/2).  The first call
   discretises from scratch (lowest index wins, no impulses); a later call with
   the same number of cells re-discretises with the first-arrival rule and
   fill/drain impulses, as a time step does. */
int orc_set_particles(orc_state *s, int np, const double *X, const double *q, const double *V,
                      const double *L) {
  int first = (s->np != np) || (s->X == NULL);
  if (first) {
    /* discard any previous cells: their nodes become resting fluid */
    double zero[3] = {0, 0, 0}, feq[NQ];
    orc_equilibrium(s->p.rho0, zero, feq);
    for (long i = 0; i < s->N; ++i)
      if (s->owner[i] >= 0) {
        s->owner[i] = FLUID;
        for (int r = 0; r < NQ; ++r) s->n[i * NQ + r] = feq[r];
      }
    free_particles(s);
    s->np = np;
    double **arrs3[] = {&s->X, &s->V, &s->L, &s->Om, &s->Fh, &s->Th, &s->Fc, &s->Tc,
                        &s->Fp, &s->Tp, &s->Fw, &s->Tw, &s->PF, &s->PT, &s->Ftot, &s->Ttot};
    for (unsigned i = 0; i < sizeof(arrs3) / sizeof(arrs3[0]); ++i)
      *arrs3[i] = (double *)xcalloc(3 * (long)np, sizeof(double));
    s->q = (double *)xcalloc(4 * (long)np, sizeof(double));
  }
  memcpy(s->X, X, sizeof(double) * 3 * np);
  memcpy(s->q, q, sizeof(double) * 4 * np);
  memcpy(s->V, V, sizeof(double) * 3 * np);
  memcpy(s->L, L, sizeof(double) * 3 * np);
  for (int k = 0; k < np; ++k) omega_from_L(&s->p, &s->q[4 * k], &s->L[3 * k], &s->Om[3 * k]);
  rediscretise(s, first);
  return 0;
}

/* ------------------------------------------------------------------ */
/* one coupled time step                                               */

/* ------------------------------------------------------------------ */
/* Lees-Edwards shear (Sec. IV, reading Q25)                           */

/* post-collision population r of fluid node src carried into a frame moving
   with du_z along z relative to the node: its equilibrium part is moved,
   n*_r + n^eq_r(rho, u + du_z e_z) - n^eq_r(rho, u) */
static double le_shifted(const orc_state *s, long src, int r, double du_z) {
  double u2[3] = {s->u[3 * src], s->u[3 * src + 1], s->u[3 * src + 2] + du_z};
  double fa[NQ], fb[NQ];
  orc_equilibrium(s->rho[src], &s->u[3 * src], fa);
  orc_equilibrium(s->rho[src], u2, fb);
  return s->nstar[src * NQ + r] + (fb[r] - fa[r]);
}

/* population r arriving at fluid node y across the plane.  Into x = 0 (c_r,x
   = +1) it comes from the image below, displaced by -D and moving with -U: its
   source is the node (nx-1, y - c_y, z - c_z + D) of this box, shifted by -U;
   into x = nx-1 (c_r,x = -1) from the image above: (0, y - c_y, z - c_z - D),
   shifted by +U.  D = U t (mod nz) falls between two nodes along z, whose
   values are interpolated linearly. */
static double le_crossing(orc_state *s, long y, int r) {
  const orc_params *p = &s->p;
  int yi = (int)((y / p->nx) % p->ny), zi = (int)(y / ((long)p->nx * p->ny));
  int up = CX[r] == 1;
  double D = fmod(s->le_U * (double)s->le_t, (double)p->nz);
  double zs = (double)(zi - CZ[r]) + (up ? D : -D);
  double z0 = floor(zs), w = zs - z0;
  int xs = up ? p->nx - 1 : 0, ys = wrap(yi - CY[r], p->ny);
  int za = (((int)z0 % p->nz) + p->nz) % p->nz, zb = (za + 1) % p->nz;
  long s0 = node_index(p, xs, ys, za), s1 = node_index(p, xs, ys, zb);
  if (s->owner[s0] != FLUID || s->owner[s1] != FLUID) s->le_bad++;
  double du = up ? -s->le_U : s->le_U;
  return (1.0 - w) * le_shifted(s, s0, r, du) + w * le_shifted(s, s1, r, du);
}

/* switch the shear on: offset U, reflection distance dr; every axis
   periodic and no wall node (the planes must hold fluid).  0 or -1. */
int orc_set_lees_edwards(orc_state *s, double U, double dr) {
  const orc_params *p = &s->p;
  if (!p->periodic[0] || !p->periodic[1] || !p->periodic[2]) return -1;
  for (long i = 0; i < s->N; ++i)
    if (IS_WALL(s->owner[i])) return -1;
  s->le_on = 1;
  s->le_U = U;
  s->le_dr = dr;
  s->le_t = 0;
  s->le_P = s->le_Psum = 0.0;
  s->le_n = s->le_reflect = s->le_bad = 0;
  return 0;
}

/* {P of the last step, P summed, steps summed, reflections, bad crossings} */
void orc_get_lees_edwards(const orc_state *s, double out[5]) {
  out[0] = s->le_P;
  out[1] = s->le_Psum;
  out[2] = (double)s->le_n;
  out[3] = (double)s->le_reflect;
  out[4] = (double)s->le_bad;
}

static void step_once(orc_state *s) {
  orc_params *p = &s->p;
  const long N = s->N;
  const double cs2 = 1.0 / 3.0;
  for (int k = 0; k < 3 * s->np; ++k)
    s->Fh[k] = s->Th[k] = s->Fc[k] = s->Tc[k] = s->Fp[k] = s->Tp[k] = s->Fw[k] = s->Tw[k] = 0.0;
  memset(s->wallmom, 0, sizeof(s->wallmom));
  s->sumC = 0.0;

  /* 1-2. moments, Guo-forced BGK collision (Eq. col, neq; reading Q1) */
  for (long i = 0; i < N; ++i) {
    if (s->owner[i] != FLUID) continue;
    double *ni = &s->n[i * NQ], *ns = &s->nstar[i * NQ];
    double rho = 0.0, j[3] = {0, 0, 0};
    for (int r = 0; r < NQ; ++r) {
      rho += ni[r];
      j[0] += ni[r] * CX[r]; j[1] += ni[r] * CY[r]; j[2] += ni[r] * CZ[r];
    }
    double Fd[3] = {rho * p->g[0], rho * p->g[1], rho * p->g[2]};
    double u[3] = {(j[0] + 0.5 * Fd[0]) / rho, (j[1] + 0.5 * Fd[1]) / rho, (j[2] + 0.5 * Fd[2]) / rho};
    double feq[NQ], S[NQ];
    orc_equilibrium(rho, u, feq);
    guo_source(u, Fd, S);
    for (int r = 0; r < NQ; ++r)
      ns[r] = ni[r] - (ni[r] - feq[r]) / p->tau + (1.0 - 1.0 / (2.0 * p->tau)) * S[r];
    s->rho[i] = rho;
    for (int k = 0; k < 3; ++k) s->u[3 * i + k] = u[k];
  }

  /* 2b. Lees-Edwards momentum transfer of this step (reading Q25): the
     z-momentum flux along +x through the plane, as the mean of its value in
     the frame below the plane and in the frame above it */
  if (s->le_on) {
    double P = 0.0;
    for (int z = 0; z < p->nz; ++z)
      for (int y = 0; y < p->ny; ++y) {
        long top = node_index(p, p->nx - 1, y, z), bot = node_index(p, 0, y, z);
        for (int r = 1; r < NQ; ++r) {
          if (CX[r] == 1 && s->owner[top] == FLUID)
            P += 0.5 * CZ[r] * (s->nstar[top * NQ + r] + le_shifted(s, top, r, -s->le_U));
          if (CX[r] == -1 && s->owner[bot] == FLUID)
            P -= 0.5 * CZ[r] * (s->nstar[bot * NQ + r] + le_shifted(s, bot, r, s->le_U));
        }
      }
    s->le_P = P;
    s->le_Psum += P;
    s->le_n++;
  }

  /* 3. contact links, Eq. (deltapppp),(deltapppm): each solid node of p with a
     neighbour owned by another cell or a wall gets -2 alpha_r rho_bar c_r */
  for (long x = 0; x < N; ++x) {
    int32_t ox = s->owner[x];
    if (ox < 0) continue;
    double xc[3];
    node_coords(p, x, xc);
    for (int r = 1; r < NQ; ++r) {
      int32_t oz = s->owner[neighbour(p, x, r, +1)];
      if (oz == FLUID || oz == ox) continue;
      double cr[3] = {CX[r], CY[r], CZ[r]};
      double f[3], arm[3], tq[3];
      for (int k = 0; k < 3; ++k) f[k] = -2.0 * weight(r) * p->rho0 * cr[k];
      for (int k = 0; k < 3; ++k) arm[k] = min_image(p, k, xc[k] + 0.5 * cr[k] - s->X[3 * ox + k]);
      cross(arm, f, tq);
      for (int k = 0; k < 3; ++k) { s->Fc[3 * ox + k] += f[k]; s->Tc[3 * ox + k] += tq[k]; }
    }
  }

  /* 4. potentials: all pairs closer than r_cut, then every cell against every
     surface wall node (a wall node linked to a non-wall node, Sec. III) */
  double *o = (double *)xcalloc(3 * (long)(s->np > 0 ? s->np : 1), sizeof(double));
  for (int k = 0; k < s->np; ++k) orc_axis(&s->q[4 * k], &o[3 * k]);
  for (int i = 0; i < s->np; ++i)
    for (int j = i + 1; j < s->np; ++j) {
      double rv[3];
      for (int k = 0; k < 3; ++k) rv[k] = min_image(p, k, s->X[3 * j + k] - s->X[3 * i + k]);
      if (dot3(rv, rv) >= p->r_cut * p->r_cut) continue;
      double Fi[3], Fj[3], Ti[3], Tj[3];
      orc_pair(p, rv, &o[3 * i], &o[3 * j], Fi, Fj, Ti, Tj);
      for (int k = 0; k < 3; ++k) {
        s->Fp[3 * i + k] += Fi[k]; s->Fp[3 * j + k] += Fj[k];
        s->Tp[3 * i + k] += Ti[k]; s->Tp[3 * j + k] += Tj[k];
      }
    }
  if (s->np > 0) {
    for (long x = 0; x < N; ++x) {
      if (!IS_WALL(s->owner[x])) continue;
      /* a surface wall node is linked to a non-wall node by some c_r (static) */
      int surface = 0;
      for (int r = 1; r < NQ && !surface; ++r) surface = !IS_WALL(s->owner[neighbour(p, x, r, +1)]);
      if (!surface) continue;
      double xc[3];
      node_coords(p, x, xc);
      for (int i = 0; i < s->np; ++i) {
        double rv[3];
        for (int k = 0; k < 3; ++k) rv[k] = min_image(p, k, xc[k] - s->X[3 * i + k]);
        double Fi[3], Ti[3];
        if (orc_wall(p, rv, &o[3 * i], Fi, Ti) > 0.0)
          for (int k = 0; k < 3; ++k) {
            s->Fp[3 * i + k] += Fi[k]; s->Tp[3 * i + k] += Ti[k];
            s->Fw[3 * i + k] += Fi[k]; s->Tw[3 * i + k] += Ti[k];
          }
      }
    }
  }
  free(o);

  /* 5. cell velocities of the half step (reading Q3).  The bounce-back
     momentum of a link (Eq. deltap) is 2 n*_rbar c_rbar minus
     w c_r (c_r . v_b) with w = 6 alpha_r rho(y) (Eq. c) and
     v_b = V + Omega x a, so the link force is linear in (V, Omega):
       F = F0 - Zff V - Zft Omega,   T = T0 - Ztf V - Ztt Omega,
     Zff = sum w c c^T, Zft = sum w c b^T, Ztf = Zft^T, Ztt = sum w b b^T,
     b = a x c_r.  The wall moves with the velocity of the step it streams
     across: V(t+1/2) and Omega(t+1/2) = I_lab(q(t))^-1 L(t+1/2) solve
       (m + Zff) V + Zft Omega = m V(t-1/2) + F0 + F_other
       Ztf V + (I_lab + Ztt) Omega = L(t-1/2) + T0 + T_other,
     with F_other, T_other the contact, potential, fill/drain and body forces. */
  double m = cell_mass(p);
  /* move_particles 2: prescribed motion, the cells keep the V and Omega of
     their last set; the forces are measured, not applied */
  if (s->np > 0 && p->move_particles == 1) {
    double *F0 = (double *)xcalloc(3 * (long)s->np, sizeof(double));
    double *T0 = (double *)xcalloc(3 * (long)s->np, sizeof(double));
    double *Z = (double *)xcalloc(36 * (long)s->np, sizeof(double)); /* 6 x 6 per cell */
    for (long y = 0; y < N; ++y) {
      if (s->owner[y] != FLUID) continue;
      double yc[3];
      node_coords(p, y, yc);
      for (int r = 1; r < NQ; ++r) {
        int32_t ox = s->owner[neighbour(p, y, r, -1)];
        if (ox < 0) continue;
        int rb = opposite(r);
        double cr[3] = {CX[r], CY[r], CZ[r]}, arm[3], b[3];
        for (int k = 0; k < 3; ++k) arm[k] = min_image(p, k, yc[k] - 0.5 * cr[k] - s->X[3 * ox + k]);
        cross(arm, cr, b);
        double nsb = s->nstar[y * NQ + rb];
        double f0[3] = {-2.0 * nsb * cr[0], -2.0 * nsb * cr[1], -2.0 * nsb * cr[2]}, t0[3];
        cross(arm, f0, t0);
        double w = 2.0 * weight(r) / cs2 * s->rho[y];
        double cb[6] = {cr[0], cr[1], cr[2], b[0], b[1], b[2]};
        for (int k = 0; k < 3; ++k) { F0[3 * ox + k] += f0[k]; T0[3 * ox + k] += t0[k]; }
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) Z[36 * ox + 6 * i + j] += w * cb[i] * cb[j];
      }
    }
    for (int i = 0; i < s->np; ++i) {
      double I[3][3], A[6][6], rhs[6], sol[6];
      inertia_lab(p, &s->q[4 * i], I);
      for (int a = 0; a < 6; ++a)
        for (int c = 0; c < 6; ++c) A[a][c] = Z[36 * i + 6 * a + c];
      for (int k = 0; k < 3; ++k) {
        A[k][k] += m;
        for (int c = 0; c < 3; ++c) A[3 + k][3 + c] += I[k][c];
        rhs[k] = m * s->V[3 * i + k] + F0[3 * i + k] + s->Fc[3 * i + k] + s->Fp[3 * i + k] + s->PF[3 * i + k] +
                 (p->body_force_on_cells ? m * p->g[k] : 0.0);
        rhs[3 + k] = s->L[3 * i + k] + T0[3 * i + k] + s->Tc[3 * i + k] + s->Tp[3 * i + k] + s->PT[3 * i + k];
      }
      solve_dense(6, A, rhs, sol);
      for (int k = 0; k < 3; ++k) {
        s->V[3 * i + k] = sol[k];
        s->Om[3 * i + k] = sol[3 + k];
      }
      for (int k = 0; k < 3; ++k) s->L[3 * i + k] = I[k][0] * sol[3] + I[k][1] * sol[4] + I[k][2] * sol[5];
    }
    free(F0); free(T0); free(Z);
  }

  /* 6. advection with mid-link bounce-back and moving-boundary term (Eq. adv,
     lbe-bb, c, lbe-bb-corr) at the cell velocities of the half step;
     momentum exchange Eq. (deltap) with reading Q7 */
  for (long y = 0; y < N; ++y) {
    if (s->owner[y] != FLUID) continue;
    double yc[3];
    node_coords(p, y, yc);
    s->nnew[y * NQ + 0] = s->nstar[y * NQ + 0];
    for (int r = 1; r < NQ; ++r) {
      long x = neighbour(p, y, r, -1); /* source node x = y - c_r */
      int32_t ox = s->owner[x];
      if (ox == FLUID) {
        int xi = (int)(y % p->nx);
        if (s->le_on && ((CX[r] == 1 && xi == 0) || (CX[r] == -1 && xi == p->nx - 1)))
          s->nnew[y * NQ + r] = le_crossing(s, y, r);
        else
          s->nnew[y * NQ + r] = s->nstar[x * NQ + r];
        continue;
      }
      int rb = opposite(r);
      double cr[3] = {CX[r], CY[r], CZ[r]};
      double vb[3] = {0, 0, 0}, arm[3] = {0, 0, 0};
      if (IS_WALL(ox)) {
        for (int k = 0; k < 3; ++k) vb[k] = p->wall_vel[WALL_ID(ox)][k];
      } else {
        /* Q2: velocity of the link midpoint y - c_r / 2, cell at X(t) */
        for (int k = 0; k < 3; ++k) arm[k] = min_image(p, k, yc[k] - 0.5 * cr[k] - s->X[3 * ox + k]);
        double w[3];
        cross(&s->Om[3 * ox], arm, w);
        for (int k = 0; k < 3; ++k) vb[k] = s->V[3 * ox + k] + w[k];
      }
      double C = 2.0 * weight(r) / cs2 * s->rho[y] * dot3(cr, vb);
      double nsb = s->nstar[y * NQ + rb];
      s->nnew[y * NQ + r] = nsb + C;
      s->sumC += C;
      double dp[3] = {(2.0 * nsb + C) * -cr[0], (2.0 * nsb + C) * -cr[1], (2.0 * nsb + C) * -cr[2]};
      if (IS_WALL(ox)) {
        for (int k = 0; k < 3; ++k) s->wallmom[WALL_ID(ox)][k] += dp[k];
      } else {
        double tq[3];
        cross(arm, dp, tq);
        for (int k = 0; k < 3; ++k) { s->Fh[3 * ox + k] += dp[k]; s->Th[3 * ox + k] += tq[k]; }
      }
    }
  }
  for (int i = 0; i < 3 * s->np; ++i) { s->Fh[i] += s->Fc[i]; s->Th[i] += s->Tc[i]; }

  /* the fluid now holds t+1 on the nodes that were fluid at t */
  for (long i = 0; i < N; ++i)
    if (s->owner[i] == FLUID)
      for (int r = 0; r < NQ; ++r) s->n[i * NQ + r] = s->nnew[i * NQ + r];

  /* totals of the step; the leap-frog moves the cells with V(t+1/2), Omega(t+1/2) */
  for (int i = 0; i < s->np; ++i) {
    for (int k = 0; k < 3; ++k) {
      s->Ftot[3 * i + k] = s->Fh[3 * i + k] + s->Fp[3 * i + k] + s->PF[3 * i + k] +
                           (p->body_force_on_cells ? m * p->g[k] : 0.0);
      s->Ttot[3 * i + k] = s->Th[3 * i + k] + s->Tp[3 * i + k] + s->PT[3 * i + k];
      s->PF[3 * i + k] = s->PT[3 * i + k] = 0.0;
    }
    /* Sec. IV: a cell whose centre is closer than le_dr to the sheared plane
       (x = -1/2, i.e. nx - 1/2) has its normal velocity negated if it moves
       toward the plane; the step's coupling used the velocity of the solve,
       the cell moves with the reflected one (reading Q25) */
    if (s->le_on && p->move_particles == 1) {
      double lo = s->X[3 * i] + 0.5, hi = (double)p->nx - 0.5 - s->X[3 * i];
      if ((lo < s->le_dr && s->V[3 * i] < 0.0) || (hi < s->le_dr && s->V[3 * i] > 0.0)) {
        s->V[3 * i] = -s->V[3 * i];
        s->le_reflect++;
      }
    }
    if (p->move_particles) rigid_advance(p, &s->X[3 * i], &s->q[4 * i], &s->V[3 * i], &s->Om[3 * i]);
  }

  /* 7. re-discretise with the first-arrival rule, fill/drain */
  if (s->np > 0 && p->move_particles) rediscretise(s, 0);
  s->t++;
  if (s->le_on) s->le_t++;
}

void orc_step(orc_state *s, int nsteps) {
  for (int k = 0; k < nsteps; ++k) step_once(s);
}

/* ------------------------------------------------------------------ */
/* read-out                                                            */

/* rho and u = (j + rho g / 2) / rho on fluid nodes; zero elsewhere */
void orc_get_fields(const orc_state *s, double *rho, double *u, int32_t *owner) {
  for (long i = 0; i < s->N; ++i) {
    if (owner) owner[i] = s->owner[i];
    if (s->owner[i] != FLUID) {
      if (rho) rho[i] = 0.0;
      if (u) u[3 * i] = u[3 * i + 1] = u[3 * i + 2] = 0.0;
      continue;
    }
    const double *ni = &s->n[i * NQ];
    double r = 0.0, j[3] = {0, 0, 0};
    for (int k = 0; k < NQ; ++k) {
      r += ni[k];
      j[0] += ni[k] * CX[k]; j[1] += ni[k] * CY[k]; j[2] += ni[k] * CZ[k];
    }
    if (rho) rho[i] = r;
    if (u)
      for (int k = 0; k < 3; ++k) u[3 * i + k] = (j[k] + 0.5 * r * s->p.g[k]) / r;
  }
}

void orc_get_populations(const orc_state *s, double *pop) { memcpy(pop, s->n, sizeof(double) * NQ * s->N); }

void orc_set_populations(orc_state *s, const double *pop) {
  for (long i = 0; i < s->N; ++i)
    for (int r = 0; r < NQ; ++r) s->n[i * NQ + r] = s->owner[i] == FLUID ? pop[i * NQ + r] : 0.0;
}

/* particle read-out: F, T = totals of the last integration; state after it */
void orc_get_particles(const orc_state *s, double *F, double *T, double *X, double *q, double *V, double *L) {
  long n3 = 3L * s->np;
  if (F) memcpy(F, s->Ftot, sizeof(double) * n3);
  if (T) memcpy(T, s->Ttot, sizeof(double) * n3);
  if (X) memcpy(X, s->X, sizeof(double) * n3);
  if (q) memcpy(q, s->q, sizeof(double) * 4 * s->np);
  if (V) memcpy(V, s->V, sizeof(double) * n3);
  if (L) memcpy(L, s->L, sizeof(double) * n3);
}

/* split of the last step's forces: link part (bounce-back + contact),
   contact part alone, potential part, angular velocity */
void orc_get_force_parts(const orc_state *s, double *Fh, double *Th, double *Fc, double *Tc, double *Fp,
                         double *Tp, double *Om) {
  long n3 = 3L * s->np;
  if (Fh) memcpy(Fh, s->Fh, sizeof(double) * n3);
  if (Th) memcpy(Th, s->Th, sizeof(double) * n3);
  if (Fc) memcpy(Fc, s->Fc, sizeof(double) * n3);
  if (Tc) memcpy(Tc, s->Tc, sizeof(double) * n3);
  if (Fp) memcpy(Fp, s->Fp, sizeof(double) * n3);
  if (Tp) memcpy(Tp, s->Tp, sizeof(double) * n3);
  if (Om) memcpy(Om, s->Om, sizeof(double) * n3);
}

/* wall-potential part of the last step's Fp, Tp (Eq. sigmaw alone) */
void orc_get_wall_parts(const orc_state *s, double *Fw, double *Tw) {
  long n3 = 3L * s->np;
  if (Fw) memcpy(Fw, s->Fw, sizeof(double) * n3);
  if (Tw) memcpy(Tw, s->Tw, sizeof(double) * n3);
}

void orc_get_pending(const orc_state *s, double *PF, double *PT) {
  long n3 = 3L * s->np;
  if (PF) memcpy(PF, s->PF, sizeof(double) * n3);
  if (PT) memcpy(PT, s->PT, sizeof(double) * n3);
}

/* counters of the last step: [sumC, mass_created, mass_deleted, n_covered,
   n_uncovered, n_switched, t], wall momentum 8 x 3 */
void orc_get_counters(const orc_state *s, double *out7, double *wallmom) {
  if (out7) {
    out7[0] = s->sumC; out7[1] = s->mass_created; out7[2] = s->mass_deleted;
    out7[3] = (double)s->n_covered; out7[4] = (double)s->n_uncovered; out7[5] = (double)s->n_switched;
    out7[6] = (double)s->t;
  }
  if (wallmom) memcpy(wallmom, s->wallmom, sizeof(s->wallmom));
}

/* boundary links: (fluid node y, direction r with y + c_r solid, owner of
   y + c_r), in (node, r) order.  Returns the count; writes at most cap. */
long orc_boundary_links(const orc_state *s, int32_t *out, long cap) {
  long k = 0;
  for (long y = 0; y < s->N; ++y) {
    if (s->owner[y] != FLUID) continue;
    for (int r = 1; r < NQ; ++r) {
      int32_t o = s->owner[neighbour(&s->p, y, r, +1)];
      if (o == FLUID) continue;
      if (k < cap) { out[3 * k] = (int32_t)y; out[3 * k + 1] = r; out[3 * k + 2] = o; }
      ++k;
    }
  }
  return k;
}

/* contact links: (node x owned by a cell, r, owner of x + c_r) where the
   neighbour is another cell or a wall, in (node, r) order */
long orc_contact_links(const orc_state *s, int32_t *out, long cap) {
  long k = 0;
  for (long x = 0; x < s->N; ++x) {
    int32_t ox = s->owner[x];
    if (ox < 0) continue;
    for (int r = 1; r < NQ; ++r) {
      int32_t o = s->owner[neighbour(&s->p, x, r, +1)];
      if (o == FLUID || o == ox) continue;
      if (k < cap) { out[3 * k] = (int32_t)x; out[3 * k + 1] = r; out[3 * k + 2] = o; }
      ++k;
    }
  }
  return k;
}

/* cell list in canonical (bin, id) order.  nb_k = max(1, floor(L_k / r_cut)),
   bin_k = floor((X_k / L_k) * nb_k) clamped to [0, nb_k - 1].
   start has nbins + 1 entries; ids has np entries.  Returns nbins. */
long orc_cell_list(const orc_state *s, int32_t *nb_out, int32_t *start, int32_t *ids) {
  const orc_params *p = &s->p;
  int n[3] = {p->nx, p->ny, p->nz}, nb[3];
  for (int k = 0; k < 3; ++k) {
    nb[k] = (int)floor((double)n[k] / p->r_cut);
    if (nb[k] < 1) nb[k] = 1;
    if (nb_out) nb_out[k] = nb[k];
  }
  long nbins = (long)nb[0] * nb[1] * nb[2];
  if (!start) return nbins;
  int32_t *bin = (int32_t *)xcalloc(s->np, sizeof(int32_t));
  for (int i = 0; i < s->np; ++i) {
    int b[3];
    for (int k = 0; k < 3; ++k) {
      b[k] = (int)floor((s->X[3 * i + k] / (double)n[k]) * (double)nb[k]);
      if (b[k] < 0) b[k] = 0;
      if (b[k] > nb[k] - 1) b[k] = nb[k] - 1;
    }
    bin[i] = b[0] + nb[0] * (b[1] + nb[1] * b[2]);
  }
  long k = 0;
  for (long b = 0; b < nbins; ++b) {
    start[b] = (int32_t)k;
    for (int i = 0; i < s->np; ++i)
      if (bin[i] == b) ids[k++] = i;
  }
  start[nbins] = (int32_t)k;
  free(bin);
  return nbins;
}

/* compensated (Neumaier) running sum, so that totals over millions of
   populations are accurate to a few ulp of the total */
typedef struct { double s, c; } ksum;
static void kadd(ksum *k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
  else k->c += (v - t) + k->s;
  k->s = t;
}

/* total fluid mass and momentum of the current populations */
void orc_totals(const orc_state *s, double *mass, double mom[3]) {
  ksum m = {0, 0}, j[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (long i = 0; i < s->N; ++i) {
    if (s->owner[i] != FLUID) continue;
    for (int r = 0; r < NQ; ++r) {
      double v = s->n[i * NQ + r];
      kadd(&m, v);
      if (CX[r]) kadd(&j[0], v * CX[r]);
      if (CY[r]) kadd(&j[1], v * CY[r]);
      if (CZ[r]) kadd(&j[2], v * CZ[r]);
    }
  }
  *mass = m.s + m.c;
  for (int k = 0; k < 3; ++k) mom[k] = j[k].s + j[k].c;
}

long orc_num_nodes(const orc_state *s) { return s->N; }
int orc_num_particles(const orc_state *s) { return s->np; }
void orc_get_owner(const orc_state *s, int32_t *owner) { memcpy(owner, s->owner, sizeof(int32_t) * s->N); }
