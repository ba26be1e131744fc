/*
 * mevp_oracle.c -- plain, serial FP64 oracle of the mEVP momentum subcycle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * What it computes (Jendersie, Lessig, Richter, "Towards a GPU-Parallelization
 * of the neXtSIM-DG Dynamical Core", PASC'24):
 *   - Eq. 2 (momentum equation) and Eq. 3 (mEVP pseudo-time iteration) on a
 *     structured quadrilateral mesh (Sec. 2.1): CG2 velocity, tensor-valued DG
 *     stress "in the gradient of the velocity space", DG ice height H and
 *     concentration A.
 *   - One subcycle is the four stages of Table 1, in that order:
 *       strain     E   = M_K^-1 sum_g w_g detJ_g phi(x_g) eps(v^{p-1})(x_g)
 *       stress     S  <- (1 - 1/alpha) S + M_K^-1 sum_g w_g detJ_g phi(x_g)
 *                         (1/alpha) s_vp(x_g)            (Listing 1 / App. A)
 *       divergence F_j = sum_K -int_K sigma(S) : grad phi_j
 *       velocity   beta-relaxed implicit update with drag and Coriolis
 *   - The stress stage follows the per-element steps of Listing 1: evaluate
 *     H, A, E at the Gauss points, clamp h, a, ice strength
 *     P = P* h exp(-C(1-a)), Delta, P/Delta, then the relaxed update with the
 *     local inverse-mass-times-weights matrix (the paper's iMJwPSI).
 *   - Element geometry (Sec. 2.1, Sec. 3.2): the bilinear map of an element's
 *     4 vertices, or the isoparametric Q2 map of its 9 CG2 node positions;
 *     J, det J and J^-1 at every quadrature point, M_K by the Gauss rule.
 *   - The transport of H and A that precedes the subcycles in every outer
 *     step (Sec. 2, Sec. 2.1): DG upwind fluxes and SSP Runge-Kutta steps.
 *
 * Everything is FP64, evaluated in the order the definitions are written,
 * compiled with -O2 -ffp-contract=off.  Per-element work is independent, so
 * the element loops may run under OpenMP without changing any result; the
 * nodal sum of element forces is always serial in ascending element order.
 *
 * Where the paper is silent (strain and divergence formulas, the velocity
 * update, the DG basis, physical constants other than P*, C, e, Delta_min)
 * this file implements the readings recorded in the project's design notes;
 * each function names the reading it follows.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)

#define MAXG 16   /* at most 4x4 Gauss points per element */
#define MAXS 8    /* at most 8 DG dofs per component     */

typedef struct {
  double Pstar;      /* ice strength parameter P* [N/m^2]                */
  double C;          /* concentration parameter in exp(-C(1-A))          */
  double e;          /* ellipse aspect ratio                             */
  double DeltaMin;   /* Delta_min [1/s]                                  */
  double alpha;      /* mEVP stress relaxation                           */
  double beta;       /* mEVP velocity relaxation                         */
  double dt;         /* outer (advection) time step [s]                  */
  double rho_ice;    /* [kg/m^3]                                         */
  double rho_water;  /* [kg/m^3]                                         */
  double Cw;         /* ocean drag coefficient                           */
  double coriolis_f; /* Coriolis parameter [1/s]                         */
} orc_params;

/* ------------------------------------------------------------------------
 * 1-D Gauss-Legendre rule on [0,1].
 * Nodes are the roots of the Legendre polynomial P_n, found by Newton's
 * method from the classical cosine initial guess; weights are the textbook
 * 2 / ((1 - x^2) P_n'(x)^2) on [-1,1], halved for [0,1].
 * ---------------------------------------------------------------------- */
static void legendre_pn(int n, double x, double *pn, double *dpn) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *pn = 1.0; *dpn = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *dpn = n * (x * p1 - p0) / (x * x - 1.0);
}

int orc_gauss(int n, double *x01, double *w01) {
  if (n < 1 || n > 4 || !x01 || !w01) return ORC_ERR_ARG;
  const double pi = 3.14159265358979323846;
  double xs[4], ws[4];
  for (int i = 0; i < n; ++i) {
    double x = cos(pi * (i + 0.75) / (n + 0.5));
    double pn = 0.0, dpn = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre_pn(n, x, &pn, &dpn);
      double dx = pn / dpn;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    legendre_pn(n, x, &pn, &dpn);
    xs[i] = x;
    ws[i] = 2.0 / ((1.0 - x * x) * dpn * dpn);
  }
  /* ascending order on [0,1] */
  for (int i = 0; i < n; ++i) {
    int k = n - 1 - i; /* cos guesses are descending */
    x01[i] = 0.5 * (1.0 + xs[k]);
    w01[i] = 0.5 * ws[k];
  }
  return ORC_OK;
}

/* Gauss points per direction for a given number of DG stress dofs (App. A:
 * 3 points for 6 or 8 dofs, 2 for 3 dofs, anything else unsupported). */
int orc_ngp(int n_s) {
  if (n_s == 6 || n_s == 8) return 3;
  if (n_s == 3) return 2;
  return -1;
}

/* ------------------------------------------------------------------------
 * DG basis on the reference square [0,1]^2: products of Legendre
 * polynomials in xh = xi - 1/2, eh = eta - 1/2 (orthogonal, so the local
 * mass matrix is diagonal on parallelograms).  Order:
 *   {1, xh, eh, xh^2 - 1/12, xh*eh, eh^2 - 1/12, (xh^2-1/12) eh, xh (eh^2-1/12)}
 * n = 1, 3, 6 or 8 takes the leading n functions.
 * ---------------------------------------------------------------------- */
int orc_dg_basis(int n, double xi, double eta, double *phi) {
  if (!(n == 1 || n == 3 || n == 6 || n == 8) || !phi) return ORC_ERR_ARG;
  double xh = xi - 0.5, eh = eta - 0.5;
  double all[8];
  all[0] = 1.0;
  all[1] = xh;
  all[2] = eh;
  all[3] = xh * xh - 1.0 / 12.0;
  all[4] = xh * eh;
  all[5] = eh * eh - 1.0 / 12.0;
  all[6] = (xh * xh - 1.0 / 12.0) * eh;
  all[7] = xh * (eh * eh - 1.0 / 12.0);
  for (int i = 0; i < n; ++i) phi[i] = all[i];
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Q2 Lagrange basis (CG2 velocity, Sec. 2.1) on [0,1]^2 with nodes
 * {0, 1/2, 1}^2; local node j = a + 3 b (a along xi, b along eta).
 * Written with the generic Lagrange product formula and its derivative.
 * ---------------------------------------------------------------------- */
static const double q2_nodes[3] = {0.0, 0.5, 1.0};

static double lagr(int a, double t) {
  double r = 1.0;
  for (int b = 0; b < 3; ++b)
    if (b != a) r *= (t - q2_nodes[b]) / (q2_nodes[a] - q2_nodes[b]);
  return r;
}

static double dlagr(int a, double t) {
  double s = 0.0;
  for (int c = 0; c < 3; ++c) {
    if (c == a) continue;
    double r = 1.0 / (q2_nodes[a] - q2_nodes[c]);
    for (int b = 0; b < 3; ++b)
      if (b != a && b != c) r *= (t - q2_nodes[b]) / (q2_nodes[a] - q2_nodes[b]);
    s += r;
  }
  return s;
}

int orc_q2_basis(double xi, double eta, double *phi, double *dxi, double *deta) {
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      int j = a + 3 * b;
      if (phi) phi[j] = lagr(a, xi) * lagr(b, eta);
      if (dxi) dxi[j] = dlagr(a, xi) * lagr(b, eta);
      if (deta) deta[j] = lagr(a, xi) * dlagr(b, eta);
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Mesh indexing: nx x ny quads, element K = ky*nx + kx; vertices
 * (nx+1)(ny+1), vertex id = jy*(nx+1) + jx, stored as (x, y) pairs;
 * CG2 nodes (2nx+1)(2ny+1), node id = iy*(2nx+1) + ix.
 * ---------------------------------------------------------------------- */
typedef struct {
  int nx, ny, n_s, n_a, ngp, ng;
  int geo;           /* 0: xy holds the vertices (bilinear Q1 element maps);
                        1: xy holds the CG2 node positions (isoparametric Q2 maps) */
  const double *xy;  /* vertices [N_v][2] or CG2 nodes [N_n][2] */
  double gx[4], gw[4];
  double psi_s[MAXS][MAXG]; /* DG stress basis at the Gauss points */
  double psi_a[MAXS][MAXG]; /* DG advection basis at the Gauss points */
  double q2[MAXG][9], q2x[MAXG][9], q2e[MAXG][9]; /* Q2 basis / reference gradients */
} mesh_t;

/* Per-element geometry: Q1 (bilinear) map from the 4 vertices, evaluated on
 * the fly (Sec. 3.2, "on-the-fly map"), its Jacobian at every Gauss point,
 * physical gradients of the Q2 basis, and the matrix
 *   iMJwPSI = M_K^{-1} [ w_g detJ_g phi_s(x_g) ]     (n_s x n_g)
 * with the local DG mass matrix M_K = sum_g w_g detJ_g phi phi^T. */
typedef struct {
  double detJ[MAXG];
  double wdet[MAXG];
  double dx[MAXG][9], dy[MAXG][9];
  double iMJwPSI[MAXS][MAXG];
  int node[9];
} elem_t;

static int invert_spd(int n, double *m /* n*n, overwritten by inverse */) {
  /* Gauss-Jordan elimination with partial pivoting. */
  double a[MAXS][2 * MAXS];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j)
      a[i][j] = (j < n) ? m[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[r][c]) > fabs(a[piv][c])) piv = r;
    if (a[piv][c] == 0.0) return ORC_ERR_ARG;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) {
        double t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t;
      }
    double d = a[c][c];
    for (int j = 0; j < 2 * n; ++j) a[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      if (f == 0.0) continue;
      for (int j = 0; j < 2 * n; ++j) a[r][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) m[i * n + j] = a[i][j + n];
  return ORC_OK;
}

static int mesh_init(mesh_t *M, int nx, int ny, const double *xy, int geo, int n_s, int n_a) {
  if (nx < 1 || ny < 1 || !xy) return ORC_ERR_ARG;
  int ngp = orc_ngp(n_s);
  if (ngp < 0) return ORC_ERR_ARG;
  if (!(n_a == 1 || n_a == 3 || n_a == 6)) return ORC_ERR_ARG;
  M->nx = nx; M->ny = ny; M->n_s = n_s; M->n_a = n_a; M->ngp = ngp; M->ng = ngp * ngp;
  M->xy = xy;
  M->geo = geo;
  orc_gauss(ngp, M->gx, M->gw);
  for (int gy = 0; gy < ngp; ++gy)
    for (int gx = 0; gx < ngp; ++gx) {
      int g = gx + ngp * gy;
      double xi = M->gx[gx], eta = M->gx[gy];
      double ps[MAXS], pa[MAXS];
      orc_dg_basis(n_s, xi, eta, ps);
      orc_dg_basis(n_a, xi, eta, pa);
      for (int s = 0; s < n_s; ++s) M->psi_s[s][g] = ps[s];
      for (int s = 0; s < n_a; ++s) M->psi_a[s][g] = pa[s];
      orc_q2_basis(xi, eta, M->q2[g], M->q2x[g], M->q2e[g]);
    }
  return ORC_OK;
}

static int elem_geometry(const mesh_t *M, int K, elem_t *E) {
  int kx = K % M->nx, ky = K / M->nx;
  int vw = M->nx + 1, nw = 2 * M->nx + 1;
  const double *x00 = M->xy + 2 * (ky * vw + kx);
  const double *x10 = M->xy + 2 * (ky * vw + kx + 1);
  const double *x01 = M->xy + 2 * ((ky + 1) * vw + kx);
  const double *x11 = M->xy + 2 * ((ky + 1) * vw + kx + 1);
  int ng = M->ng, ngp = M->ngp, n_s = M->n_s;
  for (int gy = 0; gy < ngp; ++gy)
    for (int gx = 0; gx < ngp; ++gx) {
      int g = gx + ngp * gy;
      double xi = M->gx[gx], eta = M->gx[gy];
      double J00, J01, J10, J11;
      if (M->geo) {
        /* isoparametric map: x = sum_j x_j phi_j over the 9 CG2 nodes of the
           element (Sec. 2.1: the element map from the velocity's space) */
        J00 = J01 = J10 = J11 = 0.0;
        for (int b = 0; b < 3; ++b)
          for (int a = 0; a < 3; ++a) {
            int j = a + 3 * b;
            const double *xn = M->xy + 2 * ((2 * ky + b) * nw + 2 * kx + a);
            J00 += xn[0] * M->q2x[g][j];
            J01 += xn[0] * M->q2e[g][j];
            J10 += xn[1] * M->q2x[g][j];
            J11 += xn[1] * M->q2e[g][j];
          }
      } else {
        /* derivatives of the bilinear shape functions */
        double d00x = -(1.0 - eta), d10x = (1.0 - eta), d01x = -eta, d11x = eta;
        double d00e = -(1.0 - xi), d10e = -xi, d01e = (1.0 - xi), d11e = xi;
        J00 = d00x * x00[0] + d10x * x10[0] + d01x * x01[0] + d11x * x11[0]; /* dx/dxi  */
        J01 = d00e * x00[0] + d10e * x10[0] + d01e * x01[0] + d11e * x11[0]; /* dx/deta */
        J10 = d00x * x00[1] + d10x * x10[1] + d01x * x01[1] + d11x * x11[1]; /* dy/dxi  */
        J11 = d00e * x00[1] + d10e * x10[1] + d01e * x01[1] + d11e * x11[1]; /* dy/deta */
      }
      double det = J00 * J11 - J01 * J10;
      if (!(det > 0.0)) return ORC_ERR_ARG;
      E->detJ[g] = det;
      E->wdet[g] = M->gw[gx] * M->gw[gy] * det;
      /* grad_x phi = J^{-T} grad_xi phi */
      for (int j = 0; j < 9; ++j) {
        E->dx[g][j] = (J11 * M->q2x[g][j] - J10 * M->q2e[g][j]) / det;
        E->dy[g][j] = (-J01 * M->q2x[g][j] + J00 * M->q2e[g][j]) / det;
      }
    }
  double mass[MAXS * MAXS];
  for (int s = 0; s < n_s; ++s)
    for (int t = 0; t < n_s; ++t) {
      double acc = 0.0;
      for (int g = 0; g < ng; ++g) acc += E->wdet[g] * M->psi_s[s][g] * M->psi_s[t][g];
      mass[s * n_s + t] = acc;
    }
  if (invert_spd(n_s, mass) != ORC_OK) return ORC_ERR_ARG;
  for (int s = 0; s < n_s; ++s)
    for (int g = 0; g < ng; ++g) {
      double acc = 0.0;
      for (int t = 0; t < n_s; ++t) acc += mass[s * n_s + t] * E->wdet[g] * M->psi_s[t][g];
      E->iMJwPSI[s][g] = acc;
    }
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) E->node[a + 3 * b] = (2 * ky + b) * nw + 2 * kx + a;
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Stage 1 (Table 1 "strain"): L2 projection of the symmetric velocity
 * gradient onto the DG stress space.  eps11 = du/dx, eps22 = dv/dy,
 * eps12 = (du/dy + dv/dx)/2 (tensor shear component).
 * E layout: [3][N_e][n_s] (component, element, dof; the paper's row-major
 * N x n_S matrices E11, E12, E22).  vel layout: [2][N_n].
 * ---------------------------------------------------------------------- */
static int stage_strain(const mesh_t *M, const double *vel, double *Eout) {
  int ne = M->nx * M->ny, nn = (2 * M->nx + 1) * (2 * M->ny + 1);
  int n_s = M->n_s, ng = M->ng;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int K = 0; K < ne; ++K) {
    elem_t G;
    if (elem_geometry(M, K, &G) != ORC_OK) { bad |= 1; continue; }
    double e11[MAXG], e12[MAXG], e22[MAXG];
    for (int g = 0; g < ng; ++g) {
      double ux = 0.0, uy = 0.0, vx = 0.0, vy = 0.0;
      for (int j = 0; j < 9; ++j) {
        double u = vel[G.node[j]], v = vel[nn + G.node[j]];
        ux += u * G.dx[g][j];
        uy += u * G.dy[g][j];
        vx += v * G.dx[g][j];
        vy += v * G.dy[g][j];
      }
      e11[g] = ux;
      e22[g] = vy;
      e12[g] = 0.5 * (uy + vx);
    }
    for (int s = 0; s < n_s; ++s) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int g = 0; g < ng; ++g) {
        a += G.iMJwPSI[s][g] * e11[g];
        b += G.iMJwPSI[s][g] * e12[g];
        c += G.iMJwPSI[s][g] * e22[g];
      }
      Eout[(0 * (size_t)ne + K) * n_s + s] = a;
      Eout[(1 * (size_t)ne + K) * n_s + s] = b;
      Eout[(2 * (size_t)ne + K) * n_s + s] = c;
    }
  }
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* ------------------------------------------------------------------------
 * Stage 2 (Table 1 "stress"): the mEVP stress update, Eq. 3 in the relaxation
 * form the paper's code uses, S <- (1 - 1/alpha) S + (1/alpha) M^-1 (...),
 * per element as in Listing 1 / App. A.  The viscous-plastic stress is
 * written for a general ellipse ratio e (zeta = P/(2 Delta), eta = zeta/e^2);
 * at e = 2 every coefficient equals the paper's 5/4, 3/2, 1, 5/8, 3/8, 1/4
 * exactly.  PstarK (optional, [N_e]) replaces the scalar P* of the ice
 * strength P = P* h exp(-C(1-a)) by a per-element value, the field the
 * adjoint differentiates against; NULL takes params.Pstar everywhere.
 * ---------------------------------------------------------------------- */
/* Delta = sqrt(Delta_min^2 + (1+e^-2)(e11^2+e22^2) + 2(1-e^-2) e11 e22
 *              + 4 e^-2 e12^2): 5/4, 3/2 and 1 at e = 2 (Listing 1). */
static double delta_of(const orc_params *p, double e11, double e12, double e22) {
  double ie2 = 1.0 / (p->e * p->e);
  double k_sq = 1.0 + ie2;          /* 5/4 at e = 2 */
  double k_mix = 2.0 * (1.0 - ie2); /* 3/2 */
  double k_sh = 4.0 * ie2;          /* 1   */
  return sqrt(p->DeltaMin * p->DeltaMin + k_sq * (e11 * e11 + e22 * e22) +
              k_mix * e11 * e22 + k_sh * e12 * e12);
}

static int stage_stress(const mesh_t *M, const orc_params *p, const double *Ein,
                        const double *H, const double *A, const double *PstarK, double *S) {
  int ne = M->nx * M->ny, n_s = M->n_s, n_a = M->n_a, ng = M->ng;
  double ie2 = 1.0 / (p->e * p->e);
  double c_a = 0.5 * (1.0 + ie2);   /* 5/8 */
  double c_b = 0.5 * (1.0 - ie2);   /* 3/8 */
  double c_s = ie2;                 /* 1/4 */
  double alphaInv = 1.0 / p->alpha;
  double fac = 1.0 - alphaInv;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int K = 0; K < ne; ++K) {
    elem_t G;
    if (elem_geometry(M, K, &G) != ORC_OK) { bad |= 1; continue; }
    double s11[MAXG], s12[MAXG], s22[MAXG];
    for (int g = 0; g < ng; ++g) {
      double hg = 0.0, ag = 0.0;
      for (int t = 0; t < n_a; ++t) {
        hg += H[(size_t)K * n_a + t] * M->psi_a[t][g];
        ag += A[(size_t)K * n_a + t] * M->psi_a[t][g];
      }
      double h = fmax(0.0, hg);
      double a = fmin(1.0, fmax(0.0, ag));
      /* P* is the element's own value when a per-element field is given */
      double Pst = PstarK ? PstarK[K] : p->Pstar;
      double P = Pst * h * exp(-p->C * (1.0 - a));
      double e11 = 0.0, e12 = 0.0, e22 = 0.0;
      for (int s = 0; s < n_s; ++s) {
        e11 += Ein[(0 * (size_t)ne + K) * n_s + s] * M->psi_s[s][g];
        e12 += Ein[(1 * (size_t)ne + K) * n_s + s] * M->psi_s[s][g];
        e22 += Ein[(2 * (size_t)ne + K) * n_s + s] * M->psi_s[s][g];
      }
      double delta = delta_of(p, e11, e12, e22);
      double PD = P / delta;
      s11[g] = alphaInv * (PD * (c_a * e11 + c_b * e22) - 0.5 * P);
      s12[g] = alphaInv * (PD * c_s * e12);
      s22[g] = alphaInv * (PD * (c_a * e22 + c_b * e11) - 0.5 * P);
    }
    for (int s = 0; s < n_s; ++s) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int g = 0; g < ng; ++g) {
        a += G.iMJwPSI[s][g] * s11[g];
        b += G.iMJwPSI[s][g] * s12[g];
        c += G.iMJwPSI[s][g] * s22[g];
      }
      double *q11 = &S[(0 * (size_t)ne + K) * n_s + s];
      double *q12 = &S[(1 * (size_t)ne + K) * n_s + s];
      double *q22 = &S[(2 * (size_t)ne + K) * n_s + s];
      *q11 = fac * *q11 + a;
      *q12 = fac * *q12 + b;
      *q22 = fac * *q22 + c;
    }
  }
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* ------------------------------------------------------------------------
 * Stage 3 (Table 1 "divergence"): weak divergence of the DG stress tested
 * with every CG2 basis function,
 *   f_{K,j} = - sum_g w_g detJ_g ( s11 dphi_j/dx + s12 dphi_j/dy ,
 *                                  s12 dphi_j/dx + s22 dphi_j/dy )(x_g),
 * (integration by parts of div sigma in Eq. 2; boundary nodes are Dirichlet,
 * so no boundary term), then summed to the nodes serially in ascending
 * element order, which is the fixed order SW, SE, NW, NE element of a node.
 * F layout: [2][N_n].  fel (optional) receives the per-element forces
 * [N_e][18] (x of the 9 local nodes, then y).
 * ---------------------------------------------------------------------- */
static int stage_divergence(const mesh_t *M, const double *S, double *F, double *fel) {
  int ne = M->nx * M->ny, nn = (2 * M->nx + 1) * (2 * M->ny + 1);
  int n_s = M->n_s, ng = M->ng;
  double *loc = fel ? fel : (double *)malloc(sizeof(double) * 18 * (size_t)ne);
  if (!loc) return ORC_ERR_OOM;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int K = 0; K < ne; ++K) {
    elem_t G;
    if (elem_geometry(M, K, &G) != ORC_OK) { bad |= 1; continue; }
    double g11[MAXG], g12[MAXG], g22[MAXG];
    for (int g = 0; g < ng; ++g) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int s = 0; s < n_s; ++s) {
        a += S[(0 * (size_t)ne + K) * n_s + s] * M->psi_s[s][g];
        b += S[(1 * (size_t)ne + K) * n_s + s] * M->psi_s[s][g];
        c += S[(2 * (size_t)ne + K) * n_s + s] * M->psi_s[s][g];
      }
      g11[g] = a; g12[g] = b; g22[g] = c;
    }
    for (int j = 0; j < 9; ++j) {
      double fx = 0.0, fy = 0.0;
      for (int g = 0; g < ng; ++g) {
        fx += G.wdet[g] * (g11[g] * G.dx[g][j] + g12[g] * G.dy[g][j]);
        fy += G.wdet[g] * (g12[g] * G.dx[g][j] + g22[g] * G.dy[g][j]);
      }
      loc[(size_t)K * 18 + j] = -fx;
      loc[(size_t)K * 18 + 9 + j] = -fy;
    }
  }
  if (!bad) {
    memset(F, 0, sizeof(double) * 2 * (size_t)nn);
    int nw = 2 * M->nx + 1;
    for (int K = 0; K < ne; ++K) {
      int kx = K % M->nx, ky = K / M->nx;
      for (int b = 0; b < 3; ++b)
        for (int a = 0; a < 3; ++a) {
          int j = a + 3 * b, node = (2 * ky + b) * nw + 2 * kx + a;
          F[node] += loc[(size_t)K * 18 + j];
          F[nn + node] += loc[(size_t)K * 18 + 9 + j];
        }
    }
  }
  if (!fel) free(loc);
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* ------------------------------------------------------------------------
 * Lumped nodal mass m_j = rho_ice sum_K int_K max(0, H) phi_j and lumped
 * area l_j = sum_K int_K phi_j (row sums of the CG2 mass matrices, since the
 * Q2 basis is a partition of unity), with the element Gauss rule.
 * ---------------------------------------------------------------------- */
static int lumped(const mesh_t *M, const orc_params *p, const double *H, double *m, double *l) {
  int ne = M->nx * M->ny, nn = (2 * M->nx + 1) * (2 * M->ny + 1);
  int n_a = M->n_a, ng = M->ng;
  memset(m, 0, sizeof(double) * nn);
  memset(l, 0, sizeof(double) * nn);
  for (int K = 0; K < ne; ++K) {
    elem_t G;
    if (elem_geometry(M, K, &G) != ORC_OK) return ORC_ERR_ARG;
    for (int g = 0; g < ng; ++g) {
      double hg = 0.0;
      for (int t = 0; t < n_a; ++t) hg += H[(size_t)K * n_a + t] * M->psi_a[t][g];
      double h = fmax(0.0, hg);
      for (int j = 0; j < 9; ++j) {
        m[G.node[j]] += p->rho_ice * G.wdet[g] * h * M->q2[g][j];
        l[G.node[j]] += G.wdet[g] * M->q2[g][j];
      }
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Stage 4 (Table 1 "velocity"): beta-relaxed mEVP velocity update of the
 * momentum equation (Eq. 2) at every interior CG2 node j:
 *   (m_j/dt) [ (1+beta) v^p - beta v^{p-1} - v^n ]
 *       = F_j + l_j tau_j + c_j (v_o - v^p) + m_j f (v^p_y, -v^p_x),
 *   c_j = l_j Cw rho_w |v_o - v^{p-1}|   (drag coefficient lagged),
 * solved exactly as a 2x2 system.  Boundary nodes keep v = 0 (Dirichlet).
 * A node with no mass and no drag (a = b = 0) has no defined velocity and is
 * set to 0.
 * ---------------------------------------------------------------------- */
static void stage_velocity(const mesh_t *M, const orc_params *p, const double *F,
                           const double *vprev, const double *vn, const double *tau,
                           const double *vo, const double *m, const double *l, double *vout) {
  int nw = 2 * M->nx + 1, nh = 2 * M->ny + 1, nn = nw * nh;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < nn; ++j) {
    int ix = j % nw, iy = j / nw;
    if (ix == 0 || iy == 0 || ix == nw - 1 || iy == nh - 1) {
      vout[j] = 0.0;
      vout[nn + j] = 0.0;
      continue;
    }
    double ox = vo ? vo[j] : 0.0, oy = vo ? vo[nn + j] : 0.0;
    double dvx = ox - vprev[j], dvy = oy - vprev[nn + j];
    double c = l[j] * p->Cw * p->rho_water * sqrt(dvx * dvx + dvy * dvy);
    double mdt = m[j] / p->dt;
    double a = mdt * (1.0 + p->beta) + c;
    double b = m[j] * p->coriolis_f;
    double rx = mdt * (p->beta * vprev[j] + vn[j]) + F[j] + l[j] * tau[j] + c * ox;
    double ry = mdt * (p->beta * vprev[nn + j] + vn[nn + j]) + F[nn + j] + l[j] * tau[nn + j] + c * oy;
    double det = a * a + b * b;
    if (det == 0.0) {
      vout[j] = 0.0;
      vout[nn + j] = 0.0;
      continue;
    }
    vout[j] = (a * rx + b * ry) / det;
    vout[nn + j] = (a * ry - b * rx) / det;
  }
}

static double now_s(void) {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec + 1e-9 * ts.tv_nsec;
}

/* ------------------------------------------------------------------------
 * Public entry points (ctypes).
 * ---------------------------------------------------------------------- */

/* n_sub mEVP subcycles (loop of Sec. 2: the momentum equation and the mEVP
 * iteration subcycled within one advection step, v^n and forcing fixed).
 *   vel  [2][N_n]        in: v^0 (boundary entries ignored), out: v^{n_sub}
 *   S    [3][N_e][n_s]   in/out
 *   vn   [2][N_n]        velocity at the start of the outer step
 *   tau  [2][N_n]        nodal wind stress, vo [2][N_n] or NULL (ocean at rest)
 *   E_last [3][N_e][n_s], F_last [2][N_n], fel_last [N_e][18]: optional
 *   outputs of the last subcycle; phase_sec[4] (optional) accumulates the
 *   time of strain / stress / divergence / velocity.
 *   Pstar_K [N_e] (optional): per-element ice strength parameter P* in place
 *   of params.Pstar (NULL = the scalar everywhere).                          */
int orc_subcycles(int nx, int ny, const double *xy, int geo, int n_s, int n_a, const orc_params *p,
                  const double *H, const double *A, const double *tau, const double *vo,
                  const double *vn, double *vel, double *S, int n_sub, double *E_last,
                  double *F_last, double *fel_last, double *phase_sec, const double *Pstar_K) {
  mesh_t M;
  if (!p || !H || !A || !tau || !vn || !vel || !S || n_sub < 0) return ORC_ERR_ARG;
  int rc = mesh_init(&M, nx, ny, xy, geo, n_s, n_a);
  if (rc) return rc;
  size_t ne = (size_t)nx * ny, nn = (size_t)(2 * nx + 1) * (2 * ny + 1);
  double *E = (double *)malloc(sizeof(double) * 3 * ne * n_s);
  double *F = (double *)malloc(sizeof(double) * 2 * nn);
  double *vnew = (double *)malloc(sizeof(double) * 2 * nn);
  double *m = (double *)malloc(sizeof(double) * nn);
  double *l = (double *)malloc(sizeof(double) * nn);
  if (!E || !F || !vnew || !m || !l) {
    free(E); free(F); free(vnew); free(m); free(l);
    return ORC_ERR_OOM;
  }
  rc = lumped(&M, p, H, m, l);
  for (int it = 0; it < n_sub && rc == ORC_OK; ++it) {
    int last = (it == n_sub - 1);
    double t0 = now_s();
    rc = stage_strain(&M, vel, E);
    double t1 = now_s();
    if (!rc) rc = stage_stress(&M, p, E, H, A, Pstar_K, S);
    double t2 = now_s();
    if (!rc) rc = stage_divergence(&M, S, F, last ? fel_last : NULL);
    double t3 = now_s();
    if (!rc) stage_velocity(&M, p, F, vel, vn, tau, vo, m, l, vnew);
    double t4 = now_s();
    if (!rc) memcpy(vel, vnew, sizeof(double) * 2 * nn);
    if (phase_sec) {
      phase_sec[0] += t1 - t0; phase_sec[1] += t2 - t1;
      phase_sec[2] += t3 - t2; phase_sec[3] += t4 - t3;
    }
    if (last && !rc) {
      if (E_last) memcpy(E_last, E, sizeof(double) * 3 * ne * n_s);
      if (F_last) memcpy(F_last, F, sizeof(double) * 2 * nn);
    }
  }
  free(E); free(F); free(vnew); free(m); free(l);
  return rc;
}

/* Single stages, for the pins. */
int orc_strain(int nx, int ny, const double *xy, int geo, int n_s, const double *vel, double *E) {
  mesh_t M;
  int rc = mesh_init(&M, nx, ny, xy, geo, n_s, 1);
  if (rc) return rc;
  return stage_strain(&M, vel, E);
}

int orc_stress(int nx, int ny, const double *xy, int geo, int n_s, int n_a, const orc_params *p,
               const double *E, const double *H, const double *A, double *S,
               const double *Pstar_K) {
  mesh_t M;
  int rc = mesh_init(&M, nx, ny, xy, geo, n_s, n_a);
  if (rc) return rc;
  return stage_stress(&M, p, E, H, A, Pstar_K, S);
}

/* Delta at every Gauss point, [N_e][n_g], of the strain E [3][N_e][n_s]
 * (the rheology's Delta, Listing 1, for reports of where the ice is rigid). */
int orc_delta(int nx, int ny, int n_s, const orc_params *p, const double *E, double *delta) {
  mesh_t M;
  double dummy[2] = {0.0, 0.0};
  if (!p || !E || !delta) return ORC_ERR_ARG;
  int rc = mesh_init(&M, nx, ny, dummy, 0, n_s, 1);
  if (rc) return rc;
  int ne = nx * ny, ng = M.ng;
  for (int K = 0; K < ne; ++K)
    for (int g = 0; g < ng; ++g) {
      double e11 = 0.0, e12 = 0.0, e22 = 0.0;
      for (int s = 0; s < n_s; ++s) {
        e11 += E[(0 * (size_t)ne + K) * n_s + s] * M.psi_s[s][g];
        e12 += E[(1 * (size_t)ne + K) * n_s + s] * M.psi_s[s][g];
        e22 += E[(2 * (size_t)ne + K) * n_s + s] * M.psi_s[s][g];
      }
      delta[(size_t)K * ng + g] = delta_of(p, e11, e12, e22);
    }
  return ORC_OK;
}

int orc_divergence(int nx, int ny, const double *xy, int geo, int n_s, const double *S, double *F,
                   double *fel) {
  mesh_t M;
  int rc = mesh_init(&M, nx, ny, xy, geo, n_s, 1);
  if (rc) return rc;
  return stage_divergence(&M, S, F, fel);
}

int orc_lumped(int nx, int ny, const double *xy, int geo, int n_s, int n_a, const orc_params *p,
               const double *H, double *m, double *l) {
  mesh_t M;
  int rc = mesh_init(&M, nx, ny, xy, geo, n_s, n_a);
  if (rc) return rc;
  return lumped(&M, p, H, m, l);
}

int orc_velocity(int nx, int ny, const orc_params *p, const double *F, const double *vprev,
                 const double *vn, const double *tau, const double *vo, const double *m,
                 const double *l, double *vout) {
  mesh_t M;
  if (nx < 1 || ny < 1 || !p) return ORC_ERR_ARG;
  M.nx = nx; M.ny = ny;
  stage_velocity(&M, p, F, vprev, vn, tau, vo, m, l, vout);
  return ORC_OK;
}

/* Geometry of one element for the pins: detJ and iMJwPSI at the Gauss points. */
int orc_element_map(int nx, int ny, const double *xy, int geo, int n_s, int K, double *detJ,
                    double *iMJwPSI /* n_s x n_g */) {
  mesh_t M;
  elem_t G;
  int rc = mesh_init(&M, nx, ny, xy, geo, n_s, 1);
  if (rc) return rc;
  if (K < 0 || K >= nx * ny) return ORC_ERR_ARG;
  rc = elem_geometry(&M, K, &G);
  if (rc) return rc;
  for (int g = 0; g < M.ng; ++g) {
    if (detJ) detJ[g] = G.detJ[g];
    for (int s = 0; s < n_s; ++s)
      if (iMJwPSI) iMJwPSI[s * M.ng + g] = G.iMJwPSI[s][g];
  }
  return ORC_OK;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Advection of H and A (the transport equations of Sec. 2, Eq. si:ad, with
 * zero sources), discretised as Sec. 2.1 states: discontinuous Galerkin in
 * space with the standard upwind flux, explicit Runge-Kutta in time.  The
 * paper names no flux details, quadrature or scheme order; this follows the
 * readings recorded in the design notes:
 *   - semi-discrete form on element K, test function psi_i of the n_a-dof
 *     DG space (same basis as the stress, first n_a functions):
 *       M_K dH/dt = int_K H v . grad psi_i  -  int_dK Hhat (v.n) psi_i
 *     with Hhat the trace from the element the flow leaves (upwind, chosen
 *     pointwise at each edge quadrature point); on the domain boundary the
 *     element's own trace is used both ways;
 *   - v is the CG2 velocity, held fixed over the step;
 *   - the integrals are written on the reference square with the
 *     contravariant velocity  vt = detJ J^-1 v  (vt_xi = J11 v_x - J01 v_y,
 *     vt_eta = -J10 v_x + J00 v_y), so that  int_K H v.grad psi =
 *     int_ref H (vt_xi dpsi/dxi + vt_eta dpsi/deta)  and the outward flux
 *     density per unit reference edge length is +-vt_xi on the east/west
 *     edges and +-vt_eta on the north/south edges;
 *   - quadrature: NQ x NQ Gauss points in the element and NQ on each edge,
 *     NQ = 3 for n_a = 1 or 3 and 4 for n_a = 6 (exact for every polynomial
 *     integrand of a bilinear element when the upwind side does not change
 *     along an edge);
 *   - time stepping by the strong-stability-preserving Runge-Kutta scheme of
 *     order n+1 for DG degree n: forward Euler (DG0), Heun's two-stage
 *     scheme (DG1), the Shu-Osher three-stage scheme (DG2).
 * H, A layout here: [N_e][n_a] (element-major, as in Listing 1).
 * ---------------------------------------------------------------------- */
static int adv_nq(int n_a) { return n_a == 6 ? 4 : 3; }

typedef struct {
  int nx, ny, n_a, nq;
  int geo;            /* as in mesh_t: vertices (0) or CG2 nodes (1) */
  const double *xy;
  double qx[4], qw[4];
} adv_t;

/* Jacobian of element K at reference point (xi, eta). */
static void adv_jac(const adv_t *P, int K, double xi, double eta, double J[4]) {
  int kx = K % P->nx, ky = K / P->nx, vw = P->nx + 1;
  if (P->geo) { /* isoparametric Q2 map of the 9 CG2 nodes */
    int nw = 2 * P->nx + 1;
    double dxi[9], deta[9];
    orc_q2_basis(xi, eta, NULL, dxi, deta);
    J[0] = J[1] = J[2] = J[3] = 0.0;
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        int j = a + 3 * b;
        const double *xn = P->xy + 2 * ((2 * ky + b) * nw + 2 * kx + a);
        for (int c = 0; c < 2; ++c) {
          J[2 * c + 0] += xn[c] * dxi[j];
          J[2 * c + 1] += xn[c] * deta[j];
        }
      }
    return;
  }
  const double *x00 = P->xy + 2 * (ky * vw + kx);
  const double *x10 = P->xy + 2 * (ky * vw + kx + 1);
  const double *x01 = P->xy + 2 * ((ky + 1) * vw + kx);
  const double *x11 = P->xy + 2 * ((ky + 1) * vw + kx + 1);
  for (int c = 0; c < 2; ++c) {
    J[2 * c + 0] = (1.0 - eta) * (x10[c] - x00[c]) + eta * (x11[c] - x01[c]); /* d(x_c)/dxi  */
    J[2 * c + 1] = (1.0 - xi) * (x01[c] - x00[c]) + xi * (x11[c] - x10[c]);   /* d(x_c)/deta */
  }
}

/* CG2 velocity of element K at reference point (xi, eta). */
static void adv_vel(const adv_t *P, const double *vel, int K, double xi, double eta,
                    double *vx, double *vy) {
  int kx = K % P->nx, ky = K / P->nx, nw = 2 * P->nx + 1;
  size_t nn = (size_t)nw * (2 * P->ny + 1);
  double phi[9];
  orc_q2_basis(xi, eta, phi, NULL, NULL);
  double ax = 0.0, ay = 0.0;
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      size_t node = (size_t)(2 * ky + b) * nw + 2 * kx + a;
      ax += phi[a + 3 * b] * vel[node];
      ay += phi[a + 3 * b] * vel[nn + node];
    }
  *vx = ax;
  *vy = ay;
}

/* Value of the DG field F (coefficients of element K) at (xi, eta). */
static double adv_eval(const adv_t *P, const double *F, int K, double xi, double eta) {
  double psi[MAXS];
  orc_dg_basis(P->n_a, xi, eta, psi);
  double s = 0.0;
  for (int i = 0; i < P->n_a; ++i) s += F[(size_t)K * P->n_a + i] * psi[i];
  return s;
}

/* Reference gradient of DG basis function i at (xi, eta), by the product
 * rule on the Legendre factors of orc_dg_basis. */
static void adv_dpsi(int n_a, double xi, double eta, double *dxi, double *deta) {
  double xh = xi - 0.5, eh = eta - 0.5;
  double px[3] = {1.0, xh, xh * xh - 1.0 / 12.0}, dpx[3] = {0.0, 1.0, 2.0 * xh};
  double py[3] = {1.0, eh, eh * eh - 1.0 / 12.0}, dpy[3] = {0.0, 1.0, 2.0 * eh};
  static const int kxs[8] = {0, 1, 0, 2, 1, 0, 2, 1}, kys[8] = {0, 0, 1, 0, 1, 2, 1, 2};
  for (int i = 0; i < n_a; ++i) {
    dxi[i] = dpx[kxs[i]] * py[kys[i]];
    deta[i] = px[kxs[i]] * dpy[kys[i]];
  }
}

/* L(F) = M^-1 R(F) for both fields F = H, A (same velocity, same upwind
 * decisions); out_H, out_A [N_e][n_a]. */
static int adv_operator(const adv_t *P, const double *vel, const double *H, const double *A,
                        double *out_H, double *out_A) {
  int ne = P->nx * P->ny, n_a = P->n_a, nq = P->nq;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int K = 0; K < ne; ++K) {
    int kx = K % P->nx, ky = K / P->nx;
    double RH[MAXS] = {0}, RA[MAXS] = {0}, mass[MAXS * MAXS] = {0};
    /* volume terms and the local mass matrix */
    for (int gy = 0; gy < nq; ++gy)
      for (int gx = 0; gx < nq; ++gx) {
        double xi = P->qx[gx], eta = P->qx[gy], w = P->qw[gx] * P->qw[gy];
        double J[4];
        adv_jac(P, K, xi, eta, J);
        double det = J[0] * J[3] - J[1] * J[2];
        if (!(det > 0.0)) bad |= 1;
        double vx, vy;
        adv_vel(P, vel, K, xi, eta, &vx, &vy);
        double vt_xi = J[3] * vx - J[1] * vy, vt_eta = -J[2] * vx + J[0] * vy;
        double h = adv_eval(P, H, K, xi, eta), a = adv_eval(P, A, K, xi, eta);
        double psi[MAXS], dxi[MAXS], deta[MAXS];
        orc_dg_basis(n_a, xi, eta, psi);
        adv_dpsi(n_a, xi, eta, dxi, deta);
        for (int i = 0; i < n_a; ++i) {
          double g = vt_xi * dxi[i] + vt_eta * deta[i];
          RH[i] += w * h * g;
          RA[i] += w * a * g;
          for (int j = 0; j < n_a; ++j) mass[i * n_a + j] += w * det * psi[i] * psi[j];
        }
      }
    /* edges: 0 west (xi=0), 1 east (xi=1), 2 south (eta=0), 3 north (eta=1) */
    for (int e = 0; e < 4; ++e) {
      int nb;
      if (e == 0) nb = kx > 0 ? K - 1 : -1;
      else if (e == 1) nb = kx < P->nx - 1 ? K + 1 : -1;
      else if (e == 2) nb = ky > 0 ? K - P->nx : -1;
      else nb = ky < P->ny - 1 ? K + P->nx : -1;
      for (int q = 0; q < nq; ++q) {
        double t = P->qx[q], w = P->qw[q];
        double xi, eta, nxi, neta; /* own and neighbour reference coordinates */
        if (e == 0) { xi = 0.0; eta = t; nxi = 1.0; neta = t; }
        else if (e == 1) { xi = 1.0; eta = t; nxi = 0.0; neta = t; }
        else if (e == 2) { xi = t; eta = 0.0; nxi = t; neta = 1.0; }
        else { xi = t; eta = 1.0; nxi = t; neta = 0.0; }
        double J[4];
        adv_jac(P, K, xi, eta, J);
        double vx, vy;
        adv_vel(P, vel, K, xi, eta, &vx, &vy);
        double f; /* outward flux density per unit reference length */
        if (e == 0) f = -(J[3] * vx - J[1] * vy);
        else if (e == 1) f = J[3] * vx - J[1] * vy;
        else if (e == 2) f = -(-J[2] * vx + J[0] * vy);
        else f = -J[2] * vx + J[0] * vy;
        double hh, ah;
        if (f >= 0.0 || nb < 0) {
          hh = adv_eval(P, H, K, xi, eta);
          ah = adv_eval(P, A, K, xi, eta);
        } else {
          hh = adv_eval(P, H, nb, nxi, neta);
          ah = adv_eval(P, A, nb, nxi, neta);
        }
        double psi[MAXS];
        orc_dg_basis(n_a, xi, eta, psi);
        for (int i = 0; i < n_a; ++i) {
          RH[i] -= w * f * hh * psi[i];
          RA[i] -= w * f * ah * psi[i];
        }
      }
    }
    if (invert_spd(n_a, mass) != ORC_OK) { bad |= 1; continue; }
    for (int i = 0; i < n_a; ++i) {
      double sh = 0.0, sa = 0.0;
      for (int j = 0; j < n_a; ++j) {
        sh += mass[i * n_a + j] * RH[j];
        sa += mass[i * n_a + j] * RA[j];
      }
      out_H[(size_t)K * n_a + i] = sh;
      out_A[(size_t)K * n_a + i] = sa;
    }
  }
  return bad ? ORC_ERR_ARG : ORC_OK;
}

/* n_steps advection steps of length dt (SSP Runge-Kutta of order n_a's
 * degree + 1), H and A [N_e][n_a] in/out, vel [2][N_n] fixed. */
int orc_advect(int nx, int ny, const double *xy, int geo, int n_a, const double *vel, double dt,
               int n_steps, double *H, double *A) {
  if (nx < 1 || ny < 1 || !xy || !vel || !H || !A || n_steps < 0) return ORC_ERR_ARG;
  if (!(n_a == 1 || n_a == 3 || n_a == 6)) return ORC_ERR_ARG;
  adv_t P;
  P.nx = nx; P.ny = ny; P.n_a = n_a; P.nq = adv_nq(n_a); P.xy = xy; P.geo = geo;
  orc_gauss(P.nq, P.qx, P.qw);
  size_t n = (size_t)nx * ny * n_a;
  double *LH = (double *)malloc(sizeof(double) * n), *LA = (double *)malloc(sizeof(double) * n);
  double *H1 = (double *)malloc(sizeof(double) * n), *A1 = (double *)malloc(sizeof(double) * n);
  double *H2 = (double *)malloc(sizeof(double) * n), *A2 = (double *)malloc(sizeof(double) * n);
  int rc = (LH && LA && H1 && A1 && H2 && A2) ? ORC_OK : ORC_ERR_OOM;
  for (int it = 0; it < n_steps && rc == ORC_OK; ++it) {
    /* stage 1: U1 = U + dt L(U) */
    rc = adv_operator(&P, vel, H, A, LH, LA);
    if (rc) break;
    for (size_t k = 0; k < n; ++k) { H1[k] = H[k] + dt * LH[k]; A1[k] = A[k] + dt * LA[k]; }
    if (n_a == 1) {
      memcpy(H, H1, sizeof(double) * n);
      memcpy(A, A1, sizeof(double) * n);
      continue;
    }
    rc = adv_operator(&P, vel, H1, A1, LH, LA);
    if (rc) break;
    if (n_a == 3) {
      /* Heun: U = U/2 + (U1 + dt L(U1))/2 */
      for (size_t k = 0; k < n; ++k) {
        H[k] = 0.5 * H[k] + 0.5 * (H1[k] + dt * LH[k]);
        A[k] = 0.5 * A[k] + 0.5 * (A1[k] + dt * LA[k]);
      }
      continue;
    }
    /* Shu-Osher: U2 = 3U/4 + (U1 + dt L(U1))/4, U = U/3 + 2(U2 + dt L(U2))/3 */
    for (size_t k = 0; k < n; ++k) {
      H2[k] = 0.75 * H[k] + 0.25 * (H1[k] + dt * LH[k]);
      A2[k] = 0.75 * A[k] + 0.25 * (A1[k] + dt * LA[k]);
    }
    rc = adv_operator(&P, vel, H2, A2, LH, LA);
    if (rc) break;
    for (size_t k = 0; k < n; ++k) {
      H[k] = H[k] / 3.0 + 2.0 * (H2[k] + dt * LH[k]) / 3.0;
      A[k] = A[k] / 3.0 + 2.0 * (A2[k] + dt * LA[k]) / 3.0;
    }
  }
  free(LH); free(LA); free(H1); free(A1); free(H2); free(A2);
  return rc;
}

/* The semi-discrete operator alone, L(H) = M^-1 R(H) (for the pins). */
int orc_advect_operator(int nx, int ny, const double *xy, int geo, int n_a, const double *vel,
                        const double *H, const double *A, double *LH, double *LA) {
  if (nx < 1 || ny < 1 || !xy || !vel || !H || !A || !LH || !LA) return ORC_ERR_ARG;
  if (!(n_a == 1 || n_a == 3 || n_a == 6)) return ORC_ERR_ARG;
  adv_t P;
  P.nx = nx; P.ny = ny; P.n_a = n_a; P.nq = adv_nq(n_a); P.xy = xy; P.geo = geo;
  orc_gauss(P.nq, P.qx, P.qw);
  return adv_operator(&P, vel, H, A, LH, LA);
}
