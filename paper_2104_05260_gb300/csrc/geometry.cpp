// Host FP64 geometry for HSMA (see geometry.hpp).
//
// Readings of the passages the paper leaves open (they define the method the
// library computes, so they are the same readings as the test oracle's; the
// code is independent of it):
//  * B is centred on the box centre with R_c = half the box diagonal and
//    R_s = lambda R_c (Sec. 2.2 and Sec. 3.2).
//  * Monitoring points: N_m spherical-Fibonacci points on radius R_c; 3D rows
//    impose periodicity of the potential between a point r and its wrap
//    w(r) = r - L o rnd(r/L) (rnd: half away from zero); the constant A_0^0
//    cancels and is dropped.  2D adds, on a G x G grid on each face
//    z = +-Lz/2, the dielectric Dirichlet-to-Neumann condition
//    (1 + g) dPhi/dn + (1 - g) Lambda_G Phi = 0 with Lambda_G the periodic
//    discrete DtN map, rows weighted by R_c / G (Sec. 2.2, second step).
//  * Surface charges: Q_m = sum A_nm (2n+1) R_s^(n+1) / M Y_nm(y_m/R_s) on M
//    spherical-Fibonacci points of radius R_s (Sec. 2.2, third step).
//    Option: the Fibonacci lattice rule named in Sec. 3.2 by two adjacent
//    Fibonacci numbers F_w < F (M = F): the lattice u_j = (j + 1/2)/F,
//    s_j = (j F_w mod F)/F is mapped to theta = pi psi(u), phi = 2 pi s with
//    psi(u) = u^3 (10 - 15u + 6u^2); weight w_j = 2 pi^2 psi'(u_j)
//    sin(theta_j) / F, and 1/M above becomes w_j / (4 pi).  The periodic
//    extension of the integrand in u then jumps first in its fifth
//    derivative, hence the F^-6 convergence the paper states.
//  * Image factors of Sec. 2.1, Eq. 4 with the first upper image carrying
//    gamma_top (reflection across the top interface).
#include "geometry.hpp"

#include <algorithm>
#include <cmath>
#include <complex>
#include <memory>
#include <new>

#include "../../include/hsma.h"

namespace hsma {

static const double kPi = 3.14159265358979323846;

void sphere_radius(const double box[3], double lam, double* Rc, double* Rs, double* Rs2) {
  const double a = box[0] * box[0];
  const double b = box[1] * box[1];
  const double c = box[2] * box[2];
  const double d2 = (a + b) + c;
  *Rc = 0.5 * std::sqrt(d2);
  *Rs = lam * *Rc;
  *Rs2 = *Rs * *Rs;
}

static double image_factor(int l, int sign, double gtop, double gbot) {
  const int c = (l + 1) / 2, f = l / 2;
  return sign > 0 ? std::pow(gtop, c) * std::pow(gbot, f) : std::pow(gbot, c) * std::pow(gtop, f);
}

void build_shifts(const GeoParams& gp, double Rs, std::vector<Shift>* out) {
  out->clear();
  int K[3];
  for (int d = 0; d < 3; ++d) K[d] = (int)std::ceil(Rs / gp.box[d] - 0.5);
  const double Lx = gp.box[0], Ly = gp.box[1], Lz = gp.box[2];
  out->push_back({0.0, 0.0, 1.0, 0.0, 1.0});
  if (gp.dims == 3) {
    for (int kx = -K[0]; kx <= K[0]; ++kx)
      for (int ky = -K[1]; ky <= K[1]; ++ky)
        for (int kz = -K[2]; kz <= K[2]; ++kz) {
          if (kx == 0 && ky == 0 && kz == 0) continue;
          out->push_back({kx * Lx, ky * Ly, 1.0, kz * Lz, 1.0});
        }
  } else {
    struct Layer { double zs, zo, f; };
    std::vector<Layer> layers;
    layers.push_back({1.0, 0.0, 1.0});
    for (int l = 1; l <= K[2]; ++l)
      for (int sign = 1; sign >= -1; sign -= 2) {
        const double f = image_factor(l, sign, gp.gtop, gp.gbot);
        if (f != 0.0) layers.push_back({(l % 2) ? -1.0 : 1.0, sign * (l * Lz), f});
      }
    for (int kx = -K[0]; kx <= K[0]; ++kx)
      for (int ky = -K[1]; ky <= K[1]; ++ky)
        for (size_t li = 0; li < layers.size(); ++li) {
          if (kx == 0 && ky == 0 && li == 0) continue;
          out->push_back({kx * Lx, ky * Ly, layers[li].zs, layers[li].zo, layers[li].f});
        }
  }
}

// Solid harmonics in Cartesian form.  With C_m + i S_m = (x + iy)^m and the
// polynomial U_n^m = r^(n-m) d^m P_n/dt^m (t = z/r), which obeys
//   U_m^m = (2m-1)!!,  U_{m+1}^m = (2m+1) z U_m^m,
//   (n-m) U_n^m = (2n-1) z U_{n-1}^m - (n+m-1) r^2 U_{n-2}^m,
// r^n P_n^m(cos t) cos(m f) = U_n^m C_m and the sine part is U_n^m S_m.
// The z-derivative is carried along as a dual number (C_m, S_m do not depend
// on z and d(r^2)/dz = 2z).
void solid_basis(int p, double x, double y, double z, double s, double* val, double* dz) {
  x /= s; y /= s; z /= s;
  std::vector<double> C(p + 1), S(p + 1);
  C[0] = 1.0; S[0] = 0.0;
  for (int m = 0; m < p; ++m) {
    C[m + 1] = x * C[m] - y * S[m];
    S[m + 1] = x * S[m] + y * C[m];
  }
  const double r2 = x * x + y * y + z * z, dr2 = 2.0 * z;
  const double inv4pi = 1.0 / (4.0 * kPi);
  for (int m = 0; m <= p; ++m) {
    double dfact = 1.0;
    for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
    double u2 = 0, du2 = 0, u1 = dfact, du1 = 0;
    for (int n = m; n <= p; ++n) {
      double u, du;
      if (n == m) { u = u1; du = du1; }
      else if (n == m + 1) {
        u = (2 * m + 1) * z * u1;
        du = (2 * m + 1) * (u1 + z * du1);
        u2 = u1; du2 = du1; u1 = u; du1 = du;
      } else {
        u = ((2 * n - 1) * z * u1 - (n + m - 1) * r2 * u2) / (n - m);
        du = ((2 * n - 1) * (u1 + z * du1) - (n + m - 1) * (dr2 * u2 + r2 * du2)) / (n - m);
        u2 = u1; du2 = du1; u1 = u; du1 = du;
      }
      double ratio = 1.0;  // (n-m)!/(n+m)!
      for (int k = n - m + 1; k <= n + m; ++k) ratio /= k;
      const double c = std::sqrt((2 * n + 1) * inv4pi * ratio);
      const int base = n * n + n;
      if (m == 0) {
        val[base] = c * u;
        if (dz) dz[base] = c * du / s;
      } else {
        const double cc = std::sqrt(2.0) * c;
        val[base + m] = cc * u * C[m];
        val[base - m] = cc * u * S[m];
        if (dz) {
          dz[base + m] = cc * du * C[m] / s;
          dz[base - m] = cc * du * S[m] / s;
        }
      }
    }
  }
}

// Householder QR of a tall matrix, then one-sided (Hestenes) Jacobi SVD of the
// square factor R; pinv(D) = V diag(1/sigma) (Q U_R)^T with small sigma cut.
int pseudo_inverse(const std::vector<double>& D, int m, int n, double rcond,
                   std::vector<double>* pinv, double* smax_out, double* smin_out) {
  // column-major working copy
  std::vector<double> A((size_t)m * n);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) A[i + (size_t)j * m] = D[(size_t)i * n + j];
  std::vector<double> V((size_t)m * n, 0.0);   // Householder vectors (column k from row k)
  for (int k = 0; k < n; ++k) {
    double nrm = 0;
    for (int i = k; i < m; ++i) nrm += A[i + (size_t)k * m] * A[i + (size_t)k * m];
    nrm = std::sqrt(nrm);
    const double x0 = A[k + (size_t)k * m];
    const double alpha = (x0 >= 0) ? -nrm : nrm;
    double* v = &V[(size_t)k * m];
    for (int i = k; i < m; ++i) v[i] = A[i + (size_t)k * m];
    v[k] -= alpha;
    double vn = 0;
    for (int i = k; i < m; ++i) vn += v[i] * v[i];
    vn = std::sqrt(vn);
    if (vn > 0)
      for (int i = k; i < m; ++i) v[i] /= vn;
    for (int j = k; j < n; ++j) {
      double dot = 0;
      for (int i = k; i < m; ++i) dot += v[i] * A[i + (size_t)j * m];
      for (int i = k; i < m; ++i) A[i + (size_t)j * m] -= 2.0 * v[i] * dot;
    }
  }
  // thin Q (m x n): Q = H_0 ... H_{n-1} [I; 0]
  std::vector<double> Q((size_t)m * n, 0.0);
  for (int j = 0; j < n; ++j) Q[j + (size_t)j * m] = 1.0;
  for (int k = n - 1; k >= 0; --k) {
    const double* v = &V[(size_t)k * m];
    for (int j = 0; j < n; ++j) {
      double dot = 0;
      for (int i = k; i < m; ++i) dot += v[i] * Q[i + (size_t)j * m];
      for (int i = k; i < m; ++i) Q[i + (size_t)j * m] -= 2.0 * v[i] * dot;
    }
  }
  // R (n x n), column-major
  std::vector<double> B((size_t)n * n, 0.0), Vr((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i <= j; ++i) B[i + (size_t)j * n] = A[i + (size_t)j * m];
    Vr[j + (size_t)j * n] = 1.0;
  }
  for (int sweep = 0; sweep < 80; ++sweep) {
    int rotated = 0;
    for (int i = 0; i < n - 1; ++i)
      for (int j = i + 1; j < n; ++j) {
        double a = 0, b = 0, c = 0;
        for (int k = 0; k < n; ++k) {
          const double bi = B[k + (size_t)i * n], bj = B[k + (size_t)j * n];
          a += bi * bi; b += bj * bj; c += bi * bj;
        }
        if (std::fabs(c) <= 1e-15 * std::sqrt(a * b) || c == 0.0) continue;
        ++rotated;
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int k = 0; k < n; ++k) {
          const double bi = B[k + (size_t)i * n], bj = B[k + (size_t)j * n];
          B[k + (size_t)i * n] = cs * bi - sn * bj;
          B[k + (size_t)j * n] = sn * bi + cs * bj;
          const double vi = Vr[k + (size_t)i * n], vj = Vr[k + (size_t)j * n];
          Vr[k + (size_t)i * n] = cs * vi - sn * vj;
          Vr[k + (size_t)j * n] = sn * vi + cs * vj;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> sig(n);
  double smax = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int k = 0; k < n; ++k) s += B[k + (size_t)j * n] * B[k + (size_t)j * n];
    sig[j] = std::sqrt(s);
    smax = std::max(smax, sig[j]);
  }
  const double cut = rcond * smax;
  double smin = smax;
  int rank = 0;
  // W_j = Q U_R[:, j]  (m), U_R[:, j] = B[:, j] / sigma_j
  pinv->assign((size_t)n * m, 0.0);
  std::vector<double> w(m);
  for (int j = 0; j < n; ++j) {
    if (!(sig[j] > cut)) continue;
    ++rank;
    smin = std::min(smin, sig[j]);
    for (int i = 0; i < m; ++i) {
      double s = 0;
      for (int k = 0; k < n; ++k) s += Q[i + (size_t)k * m] * B[k + (size_t)j * n];
      w[i] = s / sig[j];
    }
    // pinv += V[:, j] (1/sigma_j) w^T
    for (int r = 0; r < n; ++r) {
      const double f = Vr[r + (size_t)j * n] / sig[j];
      if (f == 0.0) continue;
      double* row = &(*pinv)[(size_t)r * m];
      for (int i = 0; i < m; ++i) row[i] += f * w[i];
    }
  }
  *smax_out = smax;
  *smin_out = smin;
  return rank;
}

static double rnd_half_away(double v) {
  return (v >= 0) ? std::floor(v + 0.5) : -std::floor(-v + 0.5);
}

static void fibonacci_sphere(int n, double R, std::vector<double>* out) {
  const double golden = (1.0 + std::sqrt(5.0)) / 2.0;
  out->resize((size_t)n * 3);
  for (int m = 0; m < n; ++m) {
    const double z = 1.0 - (2.0 * m + 1.0) / n;
    const double ph = 2.0 * kPi * m / golden;
    const double s = std::sqrt(std::max(0.0, 1.0 - z * z));
    (*out)[3 * m + 0] = R * s * std::cos(ph);
    (*out)[3 * m + 1] = R * s * std::sin(ph);
    (*out)[3 * m + 2] = R * z;
  }
}

int fibonacci_before(int M) {
  long a = 8, b = 13;
  while (b < M) {
    const long c = a + b;
    a = b;
    b = c;
  }
  return b == M ? (int)a : 0;
}

// Points of the Fibonacci lattice rule (radius R) and their weights on the
// unit sphere; M must be a Fibonacci number >= 13.
static void fibonacci_lattice(int M, double R, std::vector<double>* out, std::vector<double>* w) {
  const long Fw = fibonacci_before(M);
  out->resize((size_t)M * 3);
  w->resize(M);
  for (int j = 0; j < M; ++j) {
    const double u = (j + 0.5) / M;
    const double s = (double)(((long)j * Fw) % M) / M;
    const double psi = u * u * u * (10.0 - 15.0 * u + 6.0 * u * u);
    const double dpsi = 30.0 * u * u * (1.0 - u) * (1.0 - u);
    const double th = kPi * psi, ph = 2.0 * kPi * s;
    const double st = std::sin(th);
    (*out)[3 * j + 0] = R * st * std::cos(ph);
    (*out)[3 * j + 1] = R * st * std::sin(ph);
    (*out)[3 * j + 2] = R * std::cos(th);
    (*w)[j] = 2.0 * kPi * kPi * dpsi * st / M;
  }
}

// Periodic discrete DtN map on a G x G grid (x-major): F^-1 diag(|h|) F with
// h = 2 pi (j'/Lx, k'/Ly), j' the signed frequency.  Direct separable DFT.
struct DtN {
  int G;
  double Lx, Ly;
  std::vector<std::complex<double>> w;  // w[j*G + a] = exp(-2 pi i j a / G)
  std::vector<double> habs;
  DtN(int G_, double Lx_, double Ly_) : G(G_), Lx(Lx_), Ly(Ly_), w((size_t)G_ * G_), habs((size_t)G_ * G_) {
    for (int j = 0; j < G; ++j)
      for (int a = 0; a < G; ++a) {
        const double ang = -2.0 * kPi * (double)((long)j * a % G) / G;
        w[(size_t)j * G + a] = std::complex<double>(std::cos(ang), std::sin(ang));
      }
    for (int j = 0; j < G; ++j)
      for (int k = 0; k < G; ++k) {
        const int js = (j <= (G - 1) / 2) ? j : j - G;
        const int ks = (k <= (G - 1) / 2) ? k : k - G;
        const double hx = 2.0 * kPi * js / Lx, hy = 2.0 * kPi * ks / Ly;
        habs[(size_t)j * G + k] = std::sqrt(hx * hx + hy * hy);
      }
  }
  void apply(const double* f, double* out) const {
    std::vector<std::complex<double>> T((size_t)G * G), F((size_t)G * G);
    // along b (y)
    for (int a = 0; a < G; ++a)
      for (int k = 0; k < G; ++k) {
        std::complex<double> s = 0;
        for (int b = 0; b < G; ++b) s += f[(size_t)a * G + b] * w[(size_t)k * G + b];
        T[(size_t)a * G + k] = s;
      }
    // along a (x), multiply by |h|
    for (int j = 0; j < G; ++j)
      for (int k = 0; k < G; ++k) {
        std::complex<double> s = 0;
        for (int a = 0; a < G; ++a) s += T[(size_t)a * G + k] * w[(size_t)j * G + a];
        F[(size_t)j * G + k] = s * habs[(size_t)j * G + k];
      }
    // inverse along j then k
    for (int a = 0; a < G; ++a)
      for (int k = 0; k < G; ++k) {
        std::complex<double> s = 0;
        for (int j = 0; j < G; ++j) s += F[(size_t)j * G + k] * std::conj(w[(size_t)j * G + a]);
        T[(size_t)a * G + k] = s;
      }
    const double inv = 1.0 / ((double)G * G);
    for (int a = 0; a < G; ++a)
      for (int b = 0; b < G; ++b) {
        std::complex<double> s = 0;
        for (int k = 0; k < G; ++k) s += T[(size_t)a * G + k] * std::conj(w[(size_t)k * G + b]);
        out[(size_t)a * G + b] = s.real() * inv;
      }
  }
};

// Polynomial form: (x + iy)^m = C_m + i S_m, and V_n^m(z, r^2), the polar
// factor r^n P_n^m(cos t) / sin^m t, by the three-term recursion in n.  The
// gradient follows from dV/dz at fixed r^2, dV/d(r^2) and the x, y derivatives
// of C_m, S_m, each carried along its own recursion.
void solid_basis_grad(int p, double x, double y, double z, double s, double* val, double* grad) {
  const int nb = (p + 1) * (p + 1);
  x /= s; y /= s; z /= s;
  const double r2 = x * x + y * y + z * z;
  const double inv4pi = 1.0 / (4.0 * kPi);
  double C = 1, S = 0, Cx = 0, Cy = 0, Sx = 0, Sy = 0;
  for (int m = 0; m <= p; ++m) {
    double dfact = 1.0;
    for (int k = 2 * m - 1; k > 1; k -= 2) dfact *= k;
    double v1 = dfact, z1 = 0, q1 = 0, v2 = 0, z2 = 0, q2 = 0;  // V, dV/dz, dV/dr2
    for (int n = m; n <= p; ++n) {
      double v = v1, vz = z1, vq = q1;
      if (n == m + 1) {
        v = (2 * m + 1) * z * v1;
        vz = (2 * m + 1) * (v1 + z * z1);
        vq = (2 * m + 1) * z * q1;
      } else if (n > m + 1) {
        const double a = 2 * n - 1, b = n + m - 1;
        v = (a * z * v1 - b * r2 * v2) / (n - m);
        vz = (a * (v1 + z * z1) - b * r2 * z2) / (n - m);
        vq = (a * z * q1 - b * (v2 + r2 * q2)) / (n - m);
      }
      if (n > m) {
        v2 = v1; z2 = z1; q2 = q1;
        v1 = v; z1 = vz; q1 = vq;
      }
      double ratio = 1.0;  // (n-m)!/(n+m)!
      for (int k = n - m + 1; k <= n + m; ++k) ratio /= k;
      double c = std::sqrt((2 * n + 1) * inv4pi * ratio);
      const double Vx = 2 * x * vq, Vy = 2 * y * vq, Vz = vz + 2 * z * vq;
      const int base = n * n + n;
      if (m == 0) {
        val[base] = c * v;
        grad[base] = c * Vx / s;
        grad[nb + base] = c * Vy / s;
        grad[2 * nb + base] = c * Vz / s;
      } else {
        c *= std::sqrt(2.0);
        val[base + m] = c * v * C;
        val[base - m] = c * v * S;
        grad[base + m] = c * (Vx * C + v * Cx) / s;
        grad[base - m] = c * (Vx * S + v * Sx) / s;
        grad[nb + base + m] = c * (Vy * C + v * Cy) / s;
        grad[nb + base - m] = c * (Vy * S + v * Sy) / s;
        grad[2 * nb + base + m] = c * Vz * C / s;
        grad[2 * nb + base - m] = c * Vz * S / s;
      }
    }
    const double nC = x * C - y * S, nS = x * S + y * C;
    const double nCx = C + x * Cx - y * Sx, nSx = S + x * Sx + y * Cx;
    const double nCy = x * Cy - S - y * Sy, nSy = x * Sy + C + y * Cy;
    C = nC; S = nS; Cx = nCx; Sx = nSx; Cy = nCy; Sy = nSy;
  }
}

bool geometry_size_ok(int p, int M, int n_monitor) {
  const double nb = (double)(p + 1) * (p + 1), cap = 2147483648.0;
  return p <= 40 && (double)M * nb <= cap && (double)n_monitor * nb <= cap;
}

static int build_geometry_impl(const GeoParams& gp, Geometry* g, std::string* err) {
  const int p = gp.p, M = gp.M;
  const int nb = (p + 1) * (p + 1), nA = nb - 1;
  if (gp.dims != 2 && gp.dims != 3) { *err = "dims must be 2 or 3"; return HSMA_ERR_ARG; }
  if (p < 1 || M < nb) { *err = "need p >= 1 and M >= (p+1)^2"; return HSMA_ERR_ARG; }
  if (gp.n_monitor < nb) { *err = "n_monitor must be >= (p+1)^2"; return HSMA_ERR_ARG; }
  if (!geometry_size_ok(p, M, gp.n_monitor)) {
    *err = "need p <= 40 and M, n_monitor each at most 2^31 / (p+1)^2"; return HSMA_ERR_ARG;
  }
  if (!(gp.lam > 1.0)) { *err = "lambda must be > 1"; return HSMA_ERR_ARG; }
  for (int d = 0; d < 3; ++d)
    if (!(gp.box[d] > 0)) { *err = "box lengths must be > 0"; return HSMA_ERR_ARG; }
  if (gp.dims == 2 && (std::fabs(gp.gtop) > 1 || std::fabs(gp.gbot) > 1)) {
    *err = "|gamma| must be <= 1"; return HSMA_ERR_ARG;
  }
  if (gp.dims == 2 && gp.G < 4) { *err = "dtn_grid must be >= 4"; return HSMA_ERR_ARG; }
  if (gp.grad_rows && !(gp.grad_weight > 0.0 && std::isfinite(gp.grad_weight))) {
    *err = "grad_weight must be > 0"; return HSMA_ERR_ARG;
  }
  if (gp.surface_rule != 0 && (gp.surface_rule != 1 || fibonacci_before(M) == 0)) {
    *err = "surface_rule 1 needs M to be a Fibonacci number >= 13"; return HSMA_ERR_ARG;
  }
  g->par = gp;
  sphere_radius(gp.box, gp.lam, &g->Rc, &g->Rs, &g->Rs2);
  build_shifts(gp, g->Rs, &g->shifts);
  const double Rc = g->Rc, Rs = g->Rs;
  const double Lx = gp.box[0], Ly = gp.box[1], Lz = gp.box[2];

  // monitoring points and their wraps
  const int nm = gp.n_monitor;
  std::vector<double> mon, wrap((size_t)nm * 3);
  fibonacci_sphere(nm, Rc, &mon);
  std::vector<char> keep(nm, 1);
  for (int c = 0; c < nm; ++c) {
    for (int d = 0; d < 3; ++d) {
      const double v = mon[3 * c + d];
      wrap[3 * c + d] = (gp.dims == 2 && d == 2) ? v : v - gp.box[d] * rnd_half_away(v / gp.box[d]);
    }
    if (gp.dims == 2)
      keep[c] = (wrap[3 * c] != mon[3 * c]) || (wrap[3 * c + 1] != mon[3 * c + 1]);
  }
  g->n_mon = nm;
  const int G = gp.G;
  const int nface = (gp.dims == 2) ? G * G : 0;
  g->n_check = 2 * nm + 2 * nface;
  g->check_pts.assign((size_t)g->n_check * 3, 0.0);
  for (int c = 0; c < nm; ++c)
    for (int d = 0; d < 3; ++d) {
      g->check_pts[3 * c + d] = mon[3 * c + d];
      g->check_pts[3 * (nm + c) + d] = wrap[3 * c + d];
    }
  if (gp.dims == 2) {
    for (int f = 0; f < 2; ++f)
      for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b) {
          const size_t i = 2 * nm + (size_t)f * nface + (size_t)a * G + b;
          g->check_pts[3 * i + 0] = -0.5 * Lx + (a + 0.5) * (Lx / G);
          g->check_pts[3 * i + 1] = -0.5 * Ly + (b + 0.5) * (Ly / G);
          g->check_pts[3 * i + 2] = (f == 0) ? 0.5 * Lz : -0.5 * Lz;
        }
  }

  // design matrix D (rows x nA)
  std::vector<int> prow;  // monitoring index of each periodic row
  for (int c = 0; c < nm; ++c) if (keep[c]) prow.push_back(c);
  const int nper = (int)prow.size();
  const int rows0 = nper + 2 * nface;                       // value and DtN rows
  const int rows = rows0 + (gp.grad_rows ? 3 * nper : 0);  // + gradient rows
  std::vector<double> D((size_t)rows * nA);
  std::vector<double> bm(nb), bw(nb), dzb(nb);
  for (int r = 0; r < nper; ++r) {
    const int c = prow[r];
    solid_basis(p, mon[3 * c], mon[3 * c + 1], mon[3 * c + 2], Rc, bm.data(), nullptr);
    solid_basis(p, wrap[3 * c], wrap[3 * c + 1], wrap[3 * c + 2], Rc, bw.data(), nullptr);
    for (int k = 1; k < nb; ++k) D[(size_t)r * nA + k - 1] = bm[k] - bw[k];
  }
  const double wd = Rc / G;
  std::unique_ptr<DtN> dtn;
  if (gp.dims == 2) {
    dtn.reset(new DtN(G, Lx, Ly));
    for (int f = 0; f < 2; ++f) {
      const double gam = (f == 0) ? gp.gtop : gp.gbot;
      const double sn = (f == 0) ? 1.0 : -1.0;
      std::vector<double> Bf((size_t)nface * nb), dBf((size_t)nface * nb);
      for (int i = 0; i < nface; ++i) {
        const double* pt = &g->check_pts[3 * (2 * nm + (size_t)f * nface + i)];
        solid_basis(p, pt[0], pt[1], pt[2], Rc, &Bf[(size_t)i * nb], &dBf[(size_t)i * nb]);
      }
      std::vector<double> col(nface), lcol(nface);
      for (int k = 1; k < nb; ++k) {
        for (int i = 0; i < nface; ++i) col[i] = Bf[(size_t)i * nb + k];
        dtn->apply(col.data(), lcol.data());
        for (int i = 0; i < nface; ++i)
          D[(size_t)(nper + f * nface + i) * nA + k - 1] =
              wd * ((1.0 + gam) * sn * dBf[(size_t)i * nb + k] + (1.0 - gam) * lcol[i]);
      }
    }
  }
  // gradient-periodicity rows: component-major after all other rows
  const double wg = gp.grad_weight * Rc;
  if (gp.grad_rows) {
    std::vector<double> vm(nb), vw(nb), gm(3 * (size_t)nb), gw(3 * (size_t)nb);
    for (int r = 0; r < nper; ++r) {
      const int c = prow[r];
      solid_basis_grad(p, mon[3 * c], mon[3 * c + 1], mon[3 * c + 2], Rc, vm.data(), gm.data());
      solid_basis_grad(p, wrap[3 * c], wrap[3 * c + 1], wrap[3 * c + 2], Rc, vw.data(), gw.data());
      for (int d = 0; d < 3; ++d)
        for (int k = 1; k < nb; ++k)
          D[(size_t)(rows0 + d * nper + r) * nA + k - 1] = wg * (gm[(size_t)d * nb + k] - gw[(size_t)d * nb + k]);
    }
  }
  std::vector<double> pinv;
  g->rank = pseudo_inverse(D, rows, nA, 1e-13, &pinv, &g->smax, &g->smin);
  if (g->rank < nA) {
    *err = "fit matrix lost rank (" + std::to_string(g->rank) + " of " + std::to_string(nA) + ")";
    return HSMA_ERR_NUMERIC;
  }
  // P = pinv * S, S mapping the raw check vector v to the right-hand sides.
  g->nA = nA;
  const int nv0 = (gp.dims == 3) ? g->n_check : 2 * g->n_check;
  g->nv = nv0 + (gp.grad_rows ? 6 * nm : 0);
  g->P.assign((size_t)nA * g->nv, 0.0);
  for (int r = 0; r < nper; ++r) {
    const int c = prow[r];
    for (int k = 0; k < nA; ++k) {
      const double v = pinv[(size_t)k * rows + r];
      g->P[(size_t)k * g->nv + c] -= v;        // - Phi_B(mon)
      g->P[(size_t)k * g->nv + nm + c] += v;   // + Phi_B(wrap)
    }
  }
  if (gp.dims == 2) {
    std::vector<double> rowf(nface), lrow(nface);
    for (int f = 0; f < 2; ++f) {
      const double gam = (f == 0) ? gp.gtop : gp.gbot;
      const double sn = (f == 0) ? 1.0 : -1.0;
      const int off = 2 * nm + f * nface;
      for (int k = 0; k < nA; ++k) {
        for (int i = 0; i < nface; ++i) rowf[i] = pinv[(size_t)k * rows + nper + f * nface + i];
        dtn->apply(rowf.data(), lrow.data());   // Lambda_G is real symmetric
        for (int i = 0; i < nface; ++i) {
          g->P[(size_t)k * g->nv + off + i] += -wd * (1.0 - gam) * lrow[i];
          g->P[(size_t)k * g->nv + g->n_check + off + i] += -wd * (1.0 + gam) * sn * rowf[i];
        }
      }
    }
  }
  if (gp.grad_rows) {
    // v gains [d_x Phi_B ; d_y Phi_B ; d_z Phi_B] at [monitoring points ; wraps]
    for (int d = 0; d < 3; ++d)
      for (int r = 0; r < nper; ++r) {
        const int c = prow[r];
        for (int k = 0; k < nA; ++k) {
          const double v = wg * pinv[(size_t)k * rows + rows0 + d * nper + r];
          g->P[(size_t)k * g->nv + nv0 + 2 * nm * d + c] -= v;
          g->P[(size_t)k * g->nv + nv0 + 2 * nm * d + nm + c] += v;
        }
      }
  }
  // surface points and W
  g->W.assign((size_t)M * nA, 0.0);
  std::vector<double> fac(nb), ys(nb), wq;
  if (gp.surface_rule == 0) {
    fibonacci_sphere(M, Rs, &g->ysurf);
    for (int n = 0; n <= p; ++n)
      for (int m = -n; m <= n; ++m)
        fac[n * n + n + m] = (2 * n + 1) * std::pow(Rs, n + 1) / ((double)M * std::pow(Rc, n));
  } else {
    fibonacci_lattice(M, Rs, &g->ysurf, &wq);
    for (int n = 0; n <= p; ++n)
      for (int m = -n; m <= n; ++m)
        fac[n * n + n + m] = (2 * n + 1) * std::pow(Rs, n + 1) / (4.0 * kPi * std::pow(Rc, n));
  }
  for (int m = 0; m < M; ++m) {
    solid_basis(p, g->ysurf[3 * m], g->ysurf[3 * m + 1], g->ysurf[3 * m + 2], Rs, ys.data(), nullptr);
    const double wm = gp.surface_rule == 0 ? 1.0 : wq[m];
    for (int k = 1; k < nb; ++k)
      g->W[(size_t)m * nA + k - 1] = gp.surface_rule == 0 ? fac[k] * ys[k] : (fac[k] * ys[k]) * wm;
  }
  return HSMA_OK;
}

int build_geometry(const GeoParams& gp, Geometry* g, std::string* err) {
  try {
    return build_geometry_impl(gp, g, err);
  } catch (const std::bad_alloc&) {
    *err = "host memory ran out while building the fit operators";
    return HSMA_ERR_NOMEM;
  }
}

}  // namespace hsma
