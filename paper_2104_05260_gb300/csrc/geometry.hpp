// Host-side FP64 geometry of one HSMA set-up: everything that depends only on
// the box, the harmonic order and the point counts (the paper's "Init" step,
// Sec. 3.1): the auxiliary sphere, the image-shift table, the monitoring
// points and their wraps, the 2D face grid, the least-squares operator of
// Sec. 2.2, Eq. 6 (factored once by an SVD pseudo-inverse) and the map from
// harmonic coefficients to Fibonacci surface charges.
#pragma once

#include <string>
#include <vector>

namespace hsma {

// Image of a box-centred source (x, y, z; charge q):
//   (x + sx, y + sy, zs * z + zo), charge f * q.
struct Shift {
  double sx, sy, zs, zo, f;
};

struct GeoParams {
  int dims = 3;
  double box[3] = {1, 1, 1};
  int p = 6;
  int M = 800;
  double lam = 1.3;
  int n_monitor = 98;
  double gtop = 0, gbot = 0;
  int G = 80;
  int sphere_mask = 1;       // 0: every image of the shift table is near
  int grad_rows = 0;         // gradient-periodicity rows appended to the fit
  double grad_weight = 0.1;  // their weight, in units of R_c
  int surface_rule = 0;      // 0: golden-spiral points, equal weights; 1: Fibonacci lattice rule
};

// The Fibonacci number before M when M is a Fibonacci number >= 13 (the
// lattice rule's F_w for F = M), else 0.
int fibonacci_before(int M);

struct Geometry {
  GeoParams par;
  double Rc = 0, Rs = 0, Rs2 = 0;
  std::vector<Shift> shifts;   // identity shift first
  int n_mon = 0;
  int n_check = 0;             // targets of the check-point sum
  std::vector<double> check_pts;  // n_check * 3
  int nv = 0;                  // length of the raw check vector v
  int nA = 0;                  // (p+1)^2 - 1 fitted coefficients (n >= 1)
  std::vector<double> P;       // nA x nv, row-major: A = P v
  std::vector<double> W;       // M x nA, row-major: Q = W A
  std::vector<double> ysurf;   // M * 3
  int rank = 0;
  double smax = 0, smin = 0;
};

// R_s^2 for the sphere-membership test, in the exact FP64 operation order the
// device uses: Rc = 0.5*sqrt((Lx*Lx + Ly*Ly) + Lz*Lz), Rs = lam*Rc.
void sphere_radius(const double box[3], double lam, double* Rc, double* Rs, double* Rs2);

// Build the shift table only (identity first).
void build_shifts(const GeoParams& gp, double Rs, std::vector<Shift>* out);

// Size limits of the host-built fit operators: p <= 40, and M and
// n_monitor each times (p+1)^2 at most 2^31 entries (16 GiB of FP64).
bool geometry_size_ok(int p, int M, int n_monitor);

// Full set-up.  Returns 0, or a negative HSMA_ERR_* with *err set:
// HSMA_ERR_ARG for parameters out of range (including the size limits),
// HSMA_ERR_NOMEM when host memory runs out, HSMA_ERR_NUMERIC when the fit
// matrix loses rank.
int build_geometry(const GeoParams& gp, Geometry* g, std::string* err);

// Real orthonormal solid harmonics (r/s)^n Y_nm at (x, y, z)/s, n <= p,
// entry n*n + n + m; dz (nullable) receives d/dz of each (unscaled z).
void solid_basis(int p, double x, double y, double z, double s, double* val, double* dz);

// The same harmonics and their full gradient (unscaled coordinates):
// grad[d*(p+1)^2 + k], d = x, y, z.
void solid_basis_grad(int p, double x, double y, double z, double s, double* val, double* grad);

// Pseudo-inverse of the m x n (m >= n) row-major matrix D with relative
// singular-value cut-off rcond; pinv is n x m row-major.  Returns the rank.
int pseudo_inverse(const std::vector<double>& D, int m, int n, double rcond,
                   std::vector<double>* pinv, double* smax, double* smin);

}  // namespace hsma
