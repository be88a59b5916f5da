// Plain, slow FP64 CPU oracle for the hybrid central-moment / BGK lattice Boltzmann
// scheme for the coupled Cahn-Hilliard--Navier-Stokes equations on D2Q9
// (De Rosis, Saito, Kaneko, Abe, "Central-moments-based lattice Boltzmann scheme for
// coupled Cahn-Hilliard--Navier-Stokes equations", arXiv:1803.11345).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call this file:
// only the tests, the smoke check and the CPU-baseline leg of the benchmark do.  It shares
// no code, header, table or helper with the CUDA implementation; every constant below is
// re-typed from the paper.
//
// The scheme is executed in the paper's order, one node at a time, with no fusion:
//   stream (Eqs. 4-5) -> macroscopic rho, v, phi -> isotropic stencils (Eq. 12)
//   -> mu, p0, p~ (Eqs. 13-14 and the chemical potential in the free-energy paragraph)
//   -> f_eq, g_eq (Eqs. 8-10) -> f: central moments k = T^T f, k_eq = T^T f_eq (Eq. 15 and the
//      definition k_eq = T^T f_eq before Eq. 16), relaxation (Eq. 17), f* = (T^T)^-1 k*
//      by a numerical LU solve (no closed form) -> g: BGK (Eq. 7).
//
// Readings of the paper taken here (the paper is silent, garbled or self-contradictory):
//   * w^yy_4 = +1/3 (printed -1/3 in Eq. 11; +1/3 is the mirror image of w^xx, keeps
//     sum_i w^yy_i c_yi = 0 and reproduces the printed k_1..k_7 closed forms).
//   * k8_eq: by default the projection T^T f_eq itself (the paper defines k_eq that way);
//     k8_form = 1 uses the printed Eq. 16 term -(c_s^2/2) gamma Lap(phi) instead.
//   * omega_3 (bulk) is a free parameter; omega_6..8 default to 1 (paper) but are parameters
//     here so that the all-equal case can be compared with BGK.
//   * moving walls: halfway bounce-back, walls at y = -1/2 and y = ny - 1/2; the wall term uses
//     the boundary node's own density (f) or order parameter (g) at the colliding time level.
//   * phi at walls for the stencils: ghost rows phi(x,-1) = phi(x,0) + wet_bottom and
//     phi(x,ny) = phi(x,ny-1) + wet_top, where wet_* is the wall gradient of Eq. 18 taken along
//     the outward normal (positive: the phase phi = +1 wets the wall).  0 = mirror (neutral).
//   * body force (needed by the contact-angle test, which names a force but no forcing scheme):
//     Guo's source term S_i = w_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . F, the velocity
//     u = (sum f c + F/2) / rho, and in central-moment space k* = k + omega (k_eq - k) +
//     (1 - omega/2) T^T S for every moment (omega = 0 for k_0..k_2, so k*_1 = k_1 + F_x = F_x/2).
//     F is uniform (force_mode 0) or acts on phase l only, F (1 + phi)/2 (force_mode 1).
//   * state kept between steps = post-collision populations f*, g*.  Initialisation sets
//     f = f_eq, g = g_eq from the initial fields and applies one collision at t = 0.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// D2Q9 lattice velocities, in the order printed in the lattice paragraph before Eq. 4.
const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
// Lattice weights w_i and c_s^2 (paragraph after Eq. 14).
const double W[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                     1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
const double CS2 = 1.0 / 3.0;
// c_s^-2 = 3 exactly (c_s = 1/sqrt(3)).  Multiplying by it, rather than dividing by the rounded
// 1/3, keeps the equilibria free of a systematic 5.6e-17 relative bias.
const double INV_CS2 = 3.0;
// Surface-tension weighting factors, Eq. 11 (w^yy_4 read as +1/3, see header).
const double WXX[9] = {0, 1.0 / 3, -1.0 / 6, 1.0 / 3, -1.0 / 6,
                       -1.0 / 24, -1.0 / 24, -1.0 / 24, -1.0 / 24};
const double WYY[9] = {0, -1.0 / 6, 1.0 / 3, -1.0 / 6, 1.0 / 3,
                       -1.0 / 24, -1.0 / 24, -1.0 / 24, -1.0 / 24};
const double WXY[9] = {0, 0, 0, 0, 0, 1.0 / 4, -1.0 / 4, 1.0 / 4, -1.0 / 4};
// Isotropic stencils, Eq. 12: the weight of direction i multiplies phi(x + c_i).
const double SDX[9] = {0, 4.0 / 12, 0, -4.0 / 12, 0, 1.0 / 12, -1.0 / 12, -1.0 / 12, 1.0 / 12};
const double SDY[9] = {0, 0, 4.0 / 12, 0, -4.0 / 12, 1.0 / 12, 1.0 / 12, -1.0 / 12, -1.0 / 12};
const double SLAP[9] = {-20.0 / 6, 4.0 / 6, 4.0 / 6, 4.0 / 6, 4.0 / 6,
                        1.0 / 6, 1.0 / 6, 1.0 / 6, 1.0 / 6};

int opposite(int i) {
  for (int j = 0; j < 9; ++j)
    if (CX[j] == -CX[i] && CY[j] == -CY[i]) return j;
  return -1;
}

}  // namespace

extern "C" {

// Problem statement, in the paper's symbols.
typedef struct {
  int nx, ny;
  double tau_l, tau_g;   // f relaxation times of the phase phi=+1 (l) and phi=-1 (g); nu = c_s^2 (tau - 1/2)
  double M, Gamma;       // mobility and the free parameter Gamma: M = (1/omega_phi - 1/2) Gamma c_s^2
  double gamma, a;       // free-energy constants
  double omega3;         // bulk-viscosity relaxation of k3
  double omega6, omega7, omega8;  // higher-order relaxation (paper: 1)
  int visc_interp;       // 0: omega linear in phi (paper), 1: tau linear in phi
  int k8_form;           // 0: projection T^T f_eq, 1: printed Eq. 16
  int collision;         // 0: hybrid central moments for f (paper), 1: BGK for f (Eq. 6)
  int walls;             // 0: periodic, 1: walls at y=-1/2 and y=ny-1/2
  double u_top, u_bottom;  // x-velocity of the top / bottom wall
  double wet_bottom, wet_top;  // wall gradient of phi along the outward normal (Eq. 18)
  double Fx, Fy;         // body force per unit volume
  int force_mode;        // 0: uniform F, 1: F (1 + phi)/2 (phase l only)
} orc_params;

// ---------------------------------------------------------------------------------------
// Node-level pieces.  Each one follows a single equation of the paper.

// f equilibrium, Eq. 8 for i = 1..8 and Eq. 10 for i = 0.  pt = p~ (Eq. 14).
void orc_feq(double rho, double ux, double uy, double pt, double gx, double gy,
             double gamma, double* feq) {
  double sum = 0.0;
  double uu = ux * ux + uy * uy;
  for (int i = 1; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    feq[i] = W[i] * (INV_CS2 * pt + rho * (INV_CS2 * cu + 0.5 * INV_CS2 * INV_CS2 * cu * cu - 0.5 * INV_CS2 * uu)) +
             gamma * (WXX[i] * gx * gx + WYY[i] * gy * gy + WXY[i] * gx * gy);
    sum += feq[i];
  }
  feq[0] = rho - sum;
}

// g equilibrium, Eq. 9 for i = 1..8 and Eq. 10 for i = 0.
void orc_geq(double phi, double ux, double uy, double mu, double Gamma, double* geq) {
  double sum = 0.0;
  double uu = ux * ux + uy * uy;
  for (int i = 1; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    geq[i] = W[i] * (Gamma * mu + phi * (INV_CS2 * cu + 0.5 * INV_CS2 * INV_CS2 * cu * cu - 0.5 * INV_CS2 * uu));
    sum += geq[i];
  }
  geq[0] = phi - sum;
}

// Transformation matrix of Eq. 15, stored as T^T: row j is the basis vector T_j evaluated at the
// nine shifted velocities (c_xi - u_x, c_yi - u_y), so that k_j = sum_i TT[j][i] f_i.
void orc_basis(double ux, double uy, double* TT) {
  for (int i = 0; i < 9; ++i) {
    double X = CX[i] - ux, Y = CY[i] - uy;
    TT[0 * 9 + i] = 1.0;
    TT[1 * 9 + i] = X;
    TT[2 * 9 + i] = Y;
    TT[3 * 9 + i] = X * X + Y * Y;
    TT[4 * 9 + i] = X * X - Y * Y;
    TT[5 * 9 + i] = X * Y;
    TT[6 * 9 + i] = X * X * Y;
    TT[7 * 9 + i] = X * Y * Y;
    TT[8 * 9 + i] = X * X * Y * Y;
  }
}

// The equilibrium central moments exactly as printed (k_0..k_7 list and Eq. 16), used as an
// independent cross-check of the projection.  lap = Lap(phi).
void orc_keq_printed(double rho, double ux, double uy, double pt, double gx, double gy,
                     double lap, double gamma, double* k) {
  k[0] = rho;
  k[1] = 0.0;
  k[2] = 0.0;
  k[3] = 2.0 * pt;
  k[4] = gamma * (gx * gx - gy * gy);
  k[5] = gamma * gx * gy;
  k[6] = -0.5 * uy * k[4] - 2.0 * ux * k[5] + rho * uy * (CS2 - ux * ux) - pt * uy;
  k[7] = 0.5 * ux * k[4] - 2.0 * uy * k[5] + rho * ux * (CS2 - uy * uy) - pt * ux;
  k[8] = pt * (CS2 + ux * ux + uy * uy) - rho * CS2 * (ux * ux + uy * uy) +
         INV_CS2 * rho * ux * ux * uy * uy - CS2 / 2.0 * gamma * lap +
         0.5 * k[4] * (uy * uy - ux * ux) + 4.0 * ux * uy * k[5];
}

// Solve A x = b for a dense n x n system (n <= 9) by Gaussian elimination with partial
// pivoting.  Returns 0 on success, -1 if the matrix is singular or n is out of range.
int orc_solve(int n, const double* A_in, const double* b_in, double* x) {
  if (n < 1 || n > 9) return -1;
  double A[81], b[9];
  for (int k = 0; k < n * n; ++k) A[k] = A_in[k];
  for (int k = 0; k < n; ++k) b[k] = b_in[k];
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0) return -1;
    if (p != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[p * n + k]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < n; ++r) {
      double m = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= m * A[c * n + k];
      b[r] -= m * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
    x[r] = s / A[r * n + r];
  }
  return 0;
}

// Relaxation frequency of f for the local phi (paragraph after Eq. 14):
// omega_rho = omega_g + (phi+1)/2 (omega_l - omega_g), or the same interpolation applied to tau.
double orc_omega_rho(const orc_params* P, double phi) {
  if (P->visc_interp == 1) return 1.0 / (P->tau_g + 0.5 * (phi + 1.0) * (P->tau_l - P->tau_g));
  double wl = 1.0 / P->tau_l, wg = 1.0 / P->tau_g;
  return wg + 0.5 * (phi + 1.0) * (wl - wg);
}

// omega_phi from M = (1/omega_phi - 1/2) Gamma c_s^2 (paragraph after Eq. 14).
double orc_omega_phi(const orc_params* P) { return 1.0 / (P->M / (P->Gamma * CS2) + 0.5); }

// Wall gradient of phi for a prescribed contact angle theta (radians), Eq. 18:
// d_perp phi_w = sign(pi/2 - theta) sqrt((2a/gamma) cos(t/3) (1 - cos(t/3))), t = acos(sin^2 theta).
// The square root covers the whole product as printed; the sign (positive below 90 degrees, where
// the phase phi = +1 wets the wall) follows the paragraph after Eq. 18 on hydrophilic walls.
double orc_wall_gradient(double theta, double a, double gamma) {
  const double PI = 3.14159265358979323846;
  double st = std::sin(theta);
  double t = std::acos(st * st);
  double c = std::cos(t / 3.0);
  double mag = std::sqrt(2.0 * a / gamma * c * (1.0 - c));
  return theta < 0.5 * PI ? mag : (theta > 0.5 * PI ? -mag : 0.0);
}

// Body force at a node of order parameter phi (see the header for the two modes).
void orc_force(const orc_params* P, double phi, double* F) {
  double s = P->force_mode == 1 ? 0.5 * (1.0 + phi) : 1.0;
  F[0] = P->Fx * s;
  F[1] = P->Fy * s;
}

// Guo, Zheng & Shi (2002) forcing term for velocity u and force F:
// S_i = w_i [ (c_i - u) / c_s^2 + (c_i . u) c_i / c_s^4 ] . F.
void orc_guo_source(double ux, double uy, double Fx, double Fy, double* S) {
  for (int i = 0; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    double ax = (CX[i] - ux) * INV_CS2 + cu * CX[i] * INV_CS2 * INV_CS2;
    double ay = (CY[i] - uy) * INV_CS2 + cu * CY[i] * INV_CS2 * INV_CS2;
    S[i] = W[i] * (ax * Fx + ay * Fy);
  }
}

// Velocity of a node: (sum f c + F/2) / rho with F = orc_force(phi).
void orc_velocity(const orc_params* P, const double* f, double phi, double* u) {
  double rho = 0, jx = 0, jy = 0, F[2];
  for (int i = 0; i < 9; ++i) {
    rho += f[i];
    jx += f[i] * CX[i];
    jy += f[i] * CY[i];
  }
  orc_force(P, phi, F);
  u[0] = (jx + 0.5 * F[0]) / rho;
  u[1] = (jy + 0.5 * F[1]) / rho;
}

// Post-collision f at one node.  Central moments: Eq. 15 for the basis, k = T^T f,
// k_eq = T^T f_eq, Eq. 17 for k_3..k_8, k* = [rho, F_x/2, F_y/2, k3*..k8*] (no force: the
// paper's [rho, 0, 0, ...]), f* = (T^T)^-1 k*.  BGK (collision = 1): Eq. 6.  The force adds
// (1 - omega_j/2) (T^T S)_j to each relaxed moment, or (1 - omega/2) S_i to each BGK population.
void orc_collide_f(const orc_params* P, const double* f, double phi, double gx, double gy,
                   double lap, double* fout) {
  double rho = 0;
  for (int i = 0; i < 9; ++i) rho += f[i];
  double u[2], F[2];
  orc_velocity(P, f, phi, u);
  orc_force(P, phi, F);
  const bool forced = F[0] != 0.0 || F[1] != 0.0;
  double ux = u[0], uy = u[1];
  double S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (forced) orc_guo_source(ux, uy, F[0], F[1], S);
  double p0 = rho * CS2 + P->a * (-0.5 * phi * phi + 0.75 * phi * phi * phi * phi);  // Eq. 13
  double pt = p0 - P->gamma * phi * lap;                                              // Eq. 14
  double om = orc_omega_rho(P, phi);
  double feq[9];
  orc_feq(rho, ux, uy, pt, gx, gy, P->gamma, feq);
  if (P->collision == 1) {
    for (int i = 0; i < 9; ++i) fout[i] = f[i] + om * (feq[i] - f[i]) + (1.0 - 0.5 * om) * S[i];
    return;
  }
  double TT[81], k[9], keq[9], ks[9], kS[9];
  orc_basis(ux, uy, TT);
  for (int j = 0; j < 9; ++j) {
    k[j] = 0.0;
    keq[j] = 0.0;
    kS[j] = 0.0;
    for (int i = 0; i < 9; ++i) {
      k[j] += TT[j * 9 + i] * f[i];
      keq[j] += TT[j * 9 + i] * feq[i];
      kS[j] += TT[j * 9 + i] * S[i];
    }
  }
  if (P->k8_form == 1) {
    double kp[9];
    orc_keq_printed(rho, ux, uy, pt, gx, gy, lap, P->gamma, kp);
    keq[8] = kp[8];
  }
  const double omega[9] = {0, 0, 0, P->omega3, om, om, P->omega6, P->omega7, P->omega8};
  // Conserved moments: k_0 = rho; k_1 = sum f (c_x - u_x) = -F_x/2 before the collision and
  // gains (T^T S)_1 = F_x, so k*_1 = F_x/2 (same for y); both are 0 without a force.
  ks[0] = rho;
  ks[1] = 0.5 * F[0];
  ks[2] = 0.5 * F[1];
  for (int j = 3; j < 9; ++j) ks[j] = k[j] + omega[j] * (keq[j] - k[j]) + (1.0 - 0.5 * omega[j]) * kS[j];
  orc_solve(9, TT, ks, fout);
  // One step of iterative refinement: the elimination leaves a rounding residual with a
  // consistent sign in the momentum rows, which would make the oracle drift although k_1 and
  // k_2 are collision invariants (discussion after Eq. 17); solving for the residual once
  // removes it.
  double r[9], d[9];
  for (int j = 0; j < 9; ++j) {
    double s = ks[j];
    for (int i = 0; i < 9; ++i) s -= TT[j * 9 + i] * fout[i];
    r[j] = s;
  }
  orc_solve(9, TT, r, d);
  for (int i = 0; i < 9; ++i) fout[i] += d[i];
}

// Post-collision g at one node, Eq. 7 with g_eq from Eqs. 9-10.
void orc_collide_g(const orc_params* P, const double* g, double ux, double uy, double gx,
                   double gy, double lap, double* gout) {
  (void)gx;
  (void)gy;
  double phi = 0;
  for (int i = 0; i < 9; ++i) phi += g[i];
  double mu = P->a * (-phi + phi * phi * phi) - P->gamma * lap;  // chemical potential
  double geq[9];
  orc_geq(phi, ux, uy, mu, P->Gamma, geq);
  double wp = orc_omega_phi(P);
  for (int i = 0; i < 9; ++i) gout[i] = g[i] + wp * (geq[i] - g[i]);
}

// Stencils of Eq. 12 over a whole lattice (row-major y*nx + x).  x is periodic; y is periodic
// or, with walls, read from ghost rows phi(x,-1) = phi(x,0) + wet_bottom and
// phi(x,ny) = phi(x,ny-1) + wet_top (Eq. 18 gradients; 0 = mirror).
void orc_stencils(int nx, int ny, int walls, double wet_bottom, double wet_top, const double* phi,
                  double* gx, double* gy, double* lap) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double sx = 0, sy = 0, sl = 0;
      for (int i = 0; i < 9; ++i) {
        int xx = ((x + CX[i]) % nx + nx) % nx;
        int yy = y + CY[i];
        double ghost = 0.0;
        if (walls) {
          if (yy < 0) {
            yy = 0;
            ghost = wet_bottom;
          }
          if (yy >= ny) {
            yy = ny - 1;
            ghost = wet_top;
          }
        } else {
          yy = (yy % ny + ny) % ny;
        }
        double v = phi[(long)yy * nx + xx] + ghost;
        sx += SDX[i] * v;
        sy += SDY[i] * v;
        sl += SLAP[i] * v;
      }
      long n = (long)y * nx + x;
      gx[n] = sx;
      gy[n] = sy;
      lap[n] = sl;
    }
}

// ---------------------------------------------------------------------------------------
// Whole-lattice state: post-collision populations, nine planes each, plane i at [i*N, (i+1)*N).

typedef struct {
  orc_params P;
  long N;
  std::vector<double>* f;
  std::vector<double>* g;
} orc_state;

static void collide_all(orc_state* S, const std::vector<double>& f, const std::vector<double>& g,
                        std::vector<double>& fs, std::vector<double>& gs) {
  const orc_params* P = &S->P;
  const long N = S->N;
  std::vector<double> phi(N), gx(N), gy(N), lap(N);
  for (long n = 0; n < N; ++n) {
    double s = 0;
    for (int i = 0; i < 9; ++i) s += g[i * N + n];
    phi[n] = s;  // phi = sum_i g_i
  }
  orc_stencils(P->nx, P->ny, P->walls, P->wet_bottom, P->wet_top, phi.data(), gx.data(), gy.data(),
               lap.data());
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; ++n) {
    double fn[9], gn[9], fo[9], go[9];
    for (int i = 0; i < 9; ++i) {
      fn[i] = f[i * N + n];
      gn[i] = g[i * N + n];
    }
    double u[2];
    orc_velocity(P, fn, phi[n], u);
    orc_collide_f(P, fn, phi[n], gx[n], gy[n], lap[n], fo);
    orc_collide_g(P, gn, u[0], u[1], gx[n], gy[n], lap[n], go);
    for (int i = 0; i < 9; ++i) {
      fs[i * N + n] = fo[i];
      gs[i * N + n] = go[i];
    }
  }
}

// Streaming, Eqs. 4-5: f_i(x + c_i, t+1) = f_i*(x, t), same for g.  A link that would leave
// through a wall is reflected back to its own node in the opposite direction, with the
// moving-wall term -2 w_i s (c_i . u_w) / c_s^2, s = rho (for f) or phi (for g) of that node.
static void stream_all(const orc_state* S, const std::vector<double>& src,
                       std::vector<double>& dst, bool is_f) {
  const orc_params* P = &S->P;
  const int nx = P->nx, ny = P->ny;
  const long N = S->N;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      long n = (long)y * nx + x;
      double s = 0;
      for (int i = 0; i < 9; ++i) s += src[i * N + n];
      for (int i = 0; i < 9; ++i) {
        int xd = ((x + CX[i]) % nx + nx) % nx;
        int yd = y + CY[i];
        double v = src[i * N + n];
        if (P->walls && (yd < 0 || yd >= ny)) {
          double uw = (yd < 0) ? P->u_bottom : P->u_top;
          dst[opposite(i) * N + n] = v - 2.0 * INV_CS2 * W[i] * s * (CX[i] * uw);
          continue;
        }
        yd = (yd % ny + ny) % ny;
        dst[i * N + (long)yd * nx + xd] = v;
      }
    }
  (void)is_f;
}

void* orc_create(const orc_params* P, const double* phi0, const double* ux0, const double* uy0,
                 const double* rho0) {
  orc_state* S = new orc_state;
  S->P = *P;
  S->N = (long)P->nx * P->ny;
  const long N = S->N;
  S->f = new std::vector<double>(9 * N);
  S->g = new std::vector<double>(9 * N);
  std::vector<double> f(9 * N), g(9 * N), gx(N), gy(N), lap(N);
  orc_stencils(P->nx, P->ny, P->walls, P->wet_bottom, P->wet_top, phi0, gx.data(), gy.data(), lap.data());
  for (long n = 0; n < N; ++n) {
    double rho = rho0 ? rho0[n] : 1.0, ux = ux0 ? ux0[n] : 0.0, uy = uy0 ? uy0[n] : 0.0;
    double phi = phi0[n];
    double p0 = rho * CS2 + P->a * (-0.5 * phi * phi + 0.75 * phi * phi * phi * phi);
    double pt = p0 - P->gamma * phi * lap[n];
    double mu = P->a * (-phi + phi * phi * phi) - P->gamma * lap[n];
    double fe[9], ge[9];
    orc_feq(rho, ux, uy, pt, gx[n], gy[n], P->gamma, fe);
    orc_geq(phi, ux, uy, mu, P->Gamma, ge);
    for (int i = 0; i < 9; ++i) {
      f[i * N + n] = fe[i];
      g[i * N + n] = ge[i];
    }
  }
  collide_all(S, f, g, *S->f, *S->g);
  return S;
}

void orc_step(void* h, int nsteps) {
  orc_state* S = (orc_state*)h;
  const long N = S->N;
  std::vector<double> f(9 * N), g(9 * N);
  for (int s = 0; s < nsteps; ++s) {
    stream_all(S, *S->f, f, true);
    stream_all(S, *S->g, g, false);
    collide_all(S, f, g, *S->f, *S->g);
  }
}

// Macroscopic fields of the current (post-collision) state: rho = sum f, phi = sum g (paragraph
// after Eq. 14) and the velocity of the last collision, v = (sum f* c - F/2) / rho (the
// collision added F to sum f c, which held rho v - F/2 before it; F = 0: v = sum f c / rho).
// Any output pointer may be NULL.
void orc_fields(void* h, double* rho, double* ux, double* uy, double* phi) {
  orc_state* S = (orc_state*)h;
  const long N = S->N;
  const std::vector<double>& f = *S->f;
  const std::vector<double>& g = *S->g;
  for (long n = 0; n < N; ++n) {
    double r = 0, jx = 0, jy = 0, p = 0;
    for (int i = 0; i < 9; ++i) {
      r += f[i * N + n];
      jx += f[i * N + n] * CX[i];
      jy += f[i * N + n] * CY[i];
      p += g[i * N + n];
    }
    double F[2];
    orc_force(&S->P, p, F);
    if (rho) rho[n] = r;
    if (ux) ux[n] = (jx - 0.5 * F[0]) / r;
    if (uy) uy[n] = (jy - 0.5 * F[1]) / r;
    if (phi) phi[n] = p;
  }
}

void orc_get_populations(void* h, double* f, double* g) {
  orc_state* S = (orc_state*)h;
  std::memcpy(f, S->f->data(), sizeof(double) * 9 * S->N);
  std::memcpy(g, S->g->data(), sizeof(double) * 9 * S->N);
}

void orc_set_populations(void* h, const double* f, const double* g) {
  orc_state* S = (orc_state*)h;
  std::memcpy(S->f->data(), f, sizeof(double) * 9 * S->N);
  std::memcpy(S->g->data(), g, sizeof(double) * 9 * S->N);
}

// Compensated (Kahan) sums of phi, rho and momentum over the lattice.
void orc_sums(void* h, double* out /* [sum_phi, sum_rho, sum_jx, sum_jy] */) {
  orc_state* S = (orc_state*)h;
  const long N = S->N;
  double acc[4] = {0, 0, 0, 0}, comp[4] = {0, 0, 0, 0};
  for (long n = 0; n < N; ++n) {
    double v[4] = {0, 0, 0, 0};
    for (int i = 0; i < 9; ++i) {
      double fi = (*S->f)[i * N + n];
      v[0] += (*S->g)[i * N + n];
      v[1] += fi;
      v[2] += fi * CX[i];
      v[3] += fi * CY[i];
    }
    for (int q = 0; q < 4; ++q) {
      double yv = v[q] - comp[q];
      double t = acc[q] + yv;
      comp[q] = (t - acc[q]) - yv;
      acc[q] = t;
    }
  }
  for (int q = 0; q < 4; ++q) out[q] = acc[q];
}

// Post-collision populations of the single node (x, y) one step after the given full-lattice
// post-collision state (f, g: 9 planes of nx*ny each), computed from its neighbourhood only:
// the populations arriving at each node of the 3x3 block around (x, y) by the same streaming
// rule as stream_all (gathered instead of pushed), phi there, the Eq. 12 stencils at (x, y),
// and both collisions.  Used to check single nodes of lattices too large for a full step.
static double arriving(const orc_params* P, const double* s, long N, int x, int y, int i) {
  const int nx = P->nx, ny = P->ny;
  int ys = y - CY[i];
  if (P->walls && (ys < 0 || ys >= ny)) {
    // the population of direction opp(i) left (x, y) into the wall and came back reflected
    int j = opposite(i);
    long n = (long)y * nx + x;
    double tot = 0;
    for (int k = 0; k < 9; ++k) tot += s[k * N + n];
    double uw = (ys < 0) ? P->u_bottom : P->u_top;
    return s[j * N + n] - 2.0 * INV_CS2 * W[j] * tot * (CX[j] * uw);
  }
  ys = (ys % ny + ny) % ny;
  int xs = ((x - CX[i]) % nx + nx) % nx;
  return s[i * N + (long)ys * nx + xs];
}

void orc_node_update(const orc_params* P, const double* f, const double* g, int x, int y,
                     double* fout, double* gout) {
  const int nx = P->nx, ny = P->ny;
  const long N = (long)nx * ny;
  double phi3[3][3];
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      int xx = ((x + dx) % nx + nx) % nx;
      int yy = y + dy;
      double s = 0;
      if (P->walls) {
        if (yy < 0) {
          yy = 0;
          s = P->wet_bottom;
        }
        if (yy >= ny) {
          yy = ny - 1;
          s = P->wet_top;
        }
      } else {
        yy = (yy % ny + ny) % ny;
      }
      for (int i = 0; i < 9; ++i) s += arriving(P, g, N, xx, yy, i);
      phi3[dy + 1][dx + 1] = s;
    }
  double gxv = 0, gyv = 0, lap = 0;
  for (int i = 0; i < 9; ++i) {
    double v = phi3[CY[i] + 1][CX[i] + 1];
    gxv += SDX[i] * v;
    gyv += SDY[i] * v;
    lap += SLAP[i] * v;
  }
  double fn[9], gn[9];
  for (int i = 0; i < 9; ++i) {
    fn[i] = arriving(P, f, N, x, y, i);
    gn[i] = arriving(P, g, N, x, y, i);
  }
  double u[2];
  orc_velocity(P, fn, phi3[1][1], u);
  orc_collide_f(P, fn, phi3[1][1], gxv, gyv, lap, fout);
  orc_collide_g(P, gn, u[0], u[1], gxv, gyv, lap, gout);
}

void orc_free(void* h) {
  orc_state* S = (orc_state*)h;
  if (!S) return;
  delete S->f;
  delete S->g;
  delete S;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

}  // extern "C"
