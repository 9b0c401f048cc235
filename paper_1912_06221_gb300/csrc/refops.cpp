// Host FP64 reference operators (Sec. 3 nodal DG operators, Sec. 4.4 node reorderings,
// Sec. 4.5 reconstruction system).  Computed once per order with plain dense algebra.
#include "refops.h"

#include <cmath>
#include <cstring>
#include <mutex>
#include <memory>

namespace rdg {
namespace {

// Orthonormal Jacobi polynomials P_0..P_n^{(a,b)} at x (unit norm under (1-x)^a (1+x)^b),
// by the three-term recurrence of the normalised family.
void jacobi_all(double x, double a, double b, int n, double* P) {
  double g0 = std::pow(2.0, a + b + 1) / (a + b + 1) * std::tgamma(a + 1) * std::tgamma(b + 1) / std::tgamma(a + b + 1);
  P[0] = 1.0 / std::sqrt(g0);
  if (n == 0) return;
  double g1 = (a + 1) * (b + 1) / (a + b + 3) * g0;
  P[1] = ((a + b + 2) * x / 2 + (a - b) / 2) / std::sqrt(g1);
  double aold = 2.0 / (2 + a + b) * std::sqrt((a + 1) * (b + 1) / (a + b + 3));
  for (int i = 1; i < n; ++i) {
    double h1 = 2 * i + a + b;
    double anew = 2.0 / (h1 + 2) * std::sqrt((i + 1) * (i + 1 + a + b) * (i + 1 + a) * (i + 1 + b) / (h1 + 1) / (h1 + 3));
    double bnew = -(a * a - b * b) / h1 / (h1 + 2);
    P[i + 1] = (-aold * P[i - 1] + (x - bnew) * P[i]) / anew;
    aold = anew;
  }
}

double jacobi(double x, double a, double b, int n) {
  double P[32];
  jacobi_all(x, a, b, n, P);
  return P[n];
}

// d/dx of the orthonormal P_n^{(a,b)} = sqrt(n (n+a+b+1)) P_{n-1}^{(a+1,b+1)}
double jacobi_deriv(double x, double a, double b, int n) {
  if (n == 0) return 0.0;
  return std::sqrt(n * (n + a + b + 1)) * jacobi(x, a + 1, b + 1, n - 1);
}

// Gauss-Legendre points/weights by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 0) ? 1 : p1;
      double dp = n * (z * pn - p0) / (z * z - 1);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1, p1 = z;
    for (int k = 1; k < n; ++k) {
      double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1);
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1 - z * z) * dp * dp);
  }
}

// LGL points: -1, 1 and the roots of P_N' (Newton on P_N' using the Legendre ODE for P_N'').
std::vector<double> lgl(int N) {
  std::vector<double> t(N + 1);
  t[0] = -1;
  t[N] = 1;
  for (int i = 1; i < N; ++i) {
    double z = -std::cos(M_PI * i / N);
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 1; k < N; ++k) {
        double p2 = ((2 * k + 1) * z * p1 - k * p0) / (k + 1);
        p0 = p1;
        p1 = p2;
      }
      double dp = N * (z * p1 - p0) / (z * z - 1);
      double d2p = (2 * z * dp - N * (N + 1) * p1) / (1 - z * z);
      double dz = dp / d2p;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    t[i] = z;
  }
  return t;
}

// ---- small dense algebra (row-major) -------------------------------------------------
using Mat = std::vector<double>;

Mat matmul(const Mat& A, const Mat& B, int n, int k, int m) {
  Mat C((size_t)n * m, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < k; ++l) {
      double a = A[(size_t)i * k + l];
      for (int j = 0; j < m; ++j) C[(size_t)i * m + j] += a * B[(size_t)l * m + j];
    }
  return C;
}

Mat transpose(const Mat& A, int n, int m) {
  Mat T((size_t)n * m);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) T[(size_t)j * n + i] = A[(size_t)i * m + j];
  return T;
}

// Gauss-Jordan inverse with partial pivoting; returns false if singular.
bool invert(const Mat& A, Mat& Ai, int n) {
  Mat a = A;
  Ai.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Ai[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)p * n + c])) p = r;
    if (std::fabs(a[(size_t)p * n + c]) < 1e-300) return false;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)p * n + j], a[(size_t)c * n + j]);
        std::swap(Ai[(size_t)p * n + j], Ai[(size_t)c * n + j]);
      }
    double d = 1.0 / a[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      a[(size_t)c * n + j] *= d;
      Ai[(size_t)c * n + j] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)r * n + j] -= f * a[(size_t)c * n + j];
        Ai[(size_t)r * n + j] -= f * Ai[(size_t)c * n + j];
      }
    }
  }
  return true;
}

// Least-squares pseudo-inverse of a full-column-rank A (m x n, m >= n) by Householder QR:
// A+ = R^{-1} Q^T.  rcond receives min|R_ii| / max|R_ii|.
bool pinv_qr(const Mat& A, int m, int n, Mat& Ap, double& rcond) {
  Mat R = A;
  Mat Qt((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Qt[(size_t)i * m + i] = 1.0;
  std::vector<double> v(m);
  for (int k = 0; k < n; ++k) {
    double nrm = 0;
    for (int i = k; i < m; ++i) nrm += R[(size_t)i * n + k] * R[(size_t)i * n + k];
    nrm = std::sqrt(nrm);
    if (nrm == 0) continue;
    double alpha = R[(size_t)k * n + k] > 0 ? -nrm : nrm;
    for (int i = 0; i < m; ++i) v[i] = 0;
    for (int i = k; i < m; ++i) v[i] = R[(size_t)i * n + k];
    v[k] -= alpha;
    double vn = 0;
    for (int i = k; i < m; ++i) vn += v[i] * v[i];
    if (vn == 0) continue;
    for (int j = 0; j < n; ++j) {
      double d = 0;
      for (int i = k; i < m; ++i) d += v[i] * R[(size_t)i * n + j];
      d = 2 * d / vn;
      for (int i = k; i < m; ++i) R[(size_t)i * n + j] -= d * v[i];
    }
    for (int j = 0; j < m; ++j) {
      double d = 0;
      for (int i = k; i < m; ++i) d += v[i] * Qt[(size_t)i * m + j];
      d = 2 * d / vn;
      for (int i = k; i < m; ++i) Qt[(size_t)i * m + j] -= d * v[i];
    }
  }
  double dmin = 1e300, dmax = 0;
  for (int i = 0; i < n; ++i) {
    double d = std::fabs(R[(size_t)i * n + i]);
    dmin = std::min(dmin, d);
    dmax = std::max(dmax, d);
  }
  rcond = dmax > 0 ? dmin / dmax : 0;
  if (rcond < 1e-12) return false;
  // Ap = R1^{-1} (Qt)_{0:n, :}   (back substitution column by column)
  Ap.assign((size_t)n * m, 0.0);
  for (int c = 0; c < m; ++c) {
    for (int i = n - 1; i >= 0; --i) {
      double s = Qt[(size_t)i * m + c];
      for (int j = i + 1; j < n; ++j) s -= R[(size_t)i * n + j] * Ap[(size_t)j * m + c];
      Ap[(size_t)i * m + c] = s / R[(size_t)i * n + i];
    }
  }
  return true;
}

// ---- triangle nodes (Warp & Blend, alpha = 0) ----------------------------------------
// 1D warp: interpolant of (LGL - equidistant) on the equidistant points, evaluated at x.
double warp1d(int N, const std::vector<double>& t, double x) {
  double w = 0;
  for (int i = 0; i <= N; ++i) {
    double xi = -1.0 + 2.0 * i / N;
    double l = 1;
    for (int k = 0; k <= N; ++k)
      if (k != i) l *= (x - (-1.0 + 2.0 * k / N)) / (xi - (-1.0 + 2.0 * k / N));
    w += l * (t[i] - xi);
  }
  return w;
}

void warp_blend_nodes(int N, std::vector<double>& r, std::vector<double>& s) {
  const std::vector<double> t = lgl(N);
  const double sq3 = std::sqrt(3.0);
  r.clear();
  s.clear();
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j) {
      double L1 = double(i) / N, L3 = double(j) / N, L2 = 1 - L1 - L3;
      double x = -L2 + L3, y = (-L2 - L3 + 2 * L1) / sq3;
      auto wf = [&](double q, double Lp) {
        // edge blend 4 La Lb divided by (1 - q^2) is applied through 'Lp' = 4 La Lb
        if (std::fabs(q) >= 1 - 1e-10) return 0.0;
        return Lp * warp1d(N, t, q) / (1 - q * q);
      };
      double w1 = wf(L3 - L2, 4 * L2 * L3);
      double w2 = wf(L1 - L3, 4 * L1 * L3);
      double w3 = wf(L2 - L1, 4 * L1 * L2);
      x += w1 + std::cos(2 * M_PI / 3) * w2 + std::cos(4 * M_PI / 3) * w3;
      y += std::sin(2 * M_PI / 3) * w2 + std::sin(4 * M_PI / 3) * w3;
      double l1 = (sq3 * y + 1) / 3, l2 = (-3 * x - sq3 * y + 2) / 6, l3 = (3 * x - sq3 * y + 2) / 6;
      r.push_back(-l2 + l3 - l1);
      s.push_back(-l2 - l3 + l1);
    }
}

double legn(int n, double x) { return jacobi(x, 0, 0, n); }
double dlegn(int n, double x) { return jacobi_deriv(x, 0, 0, n); }

std::unique_ptr<RefOps> build(int N, const char** err) {
  auto o = std::make_unique<RefOps>();
  o->N = N;
  const int Np = o->Np = np_of(N), Nfp = o->Nfp = nfp_of(N), Mp = o->Mp = mp_of(N);
  warp_blend_nodes(N, o->r, o->s);
  Mat Vr((size_t)Np * Np), Vs((size_t)Np * Np);
  o->V.resize((size_t)Np * Np);
  for (int i = 0; i < Np; ++i)
    simplex_basis(N, o->r[i], o->s[i], &o->V[(size_t)i * Np], &Vr[(size_t)i * Np], &Vs[(size_t)i * Np]);
  if (!invert(o->V, o->Vinv, Np)) { *err = "Vandermonde matrix singular"; return nullptr; }
  o->Dr = matmul(Vr, o->Vinv, Np, Np, Np);
  o->Ds = matmul(Vs, o->Vinv, Np, Np, Np);
  Mat Minv = matmul(o->V, transpose(o->V, Np, Np), Np, Np, Np);
  if (!invert(Minv, o->M, Np)) { *err = "mass matrix singular"; return nullptr; }
  o->Wr = matmul(matmul(Minv, transpose(o->Dr, Np, Np), Np, Np, Np), o->M, Np, Np, Np);
  o->Ws = matmul(matmul(Minv, transpose(o->Ds, Np, Np), Np, Np, Np), o->M, Np, Np, Np);
  // face masks (counter-clockwise along faces v1->v2, v2->v3, v3->v1)
  std::vector<int> idx((N + 1) * (N + 1), -1);
  {
    int k = 0;
    for (int i = 0; i <= N; ++i)
      for (int j = 0; j <= N - i; ++j) idx[i * (N + 1) + j] = k++;
  }
  o->Fmask.resize(3 * Nfp);
  for (int q = 0; q <= N; ++q) {
    o->Fmask[0 * Nfp + q] = idx[0 * (N + 1) + q];
    o->Fmask[1 * Nfp + q] = idx[q * (N + 1) + (N - q)];
    o->Fmask[2 * Nfp + q] = idx[(N - q) * (N + 1) + 0];
  }
  // face mass on the LGL points and LIFT = M^{-1} E
  std::vector<double> t = lgl(N);
  Mat V1((size_t)Nfp * Nfp);
  for (int i = 0; i < Nfp; ++i)
    for (int j = 0; j < Nfp; ++j) V1[(size_t)i * Nfp + j] = legn(j, t[i]);
  Mat M1inv = matmul(V1, transpose(V1, Nfp, Nfp), Nfp, Nfp, Nfp), M1;
  if (!invert(M1inv, M1, Nfp)) { *err = "face mass singular"; return nullptr; }
  Mat E((size_t)Np * 3 * Nfp, 0.0);
  for (int f = 0; f < 3; ++f)
    for (int a = 0; a < Nfp; ++a)
      for (int q = 0; q < Nfp; ++q) E[(size_t)o->Fmask[f * Nfp + a] * 3 * Nfp + f * Nfp + q] = M1[(size_t)a * Nfp + q];
  o->LIFT = matmul(Minv, E, Np, Np, 3 * Nfp);
  // node permutations of the three orderings that put face f on the hypotenuse (Sec. 4.4)
  o->perm.assign(3 * Np, -1);
  const int fa[3] = {0, 1, 2}, fb[3] = {1, 2, 0};
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < Np; ++i) {
      double lam[3] = {-(o->r[i] + o->s[i]) / 2, (o->r[i] + 1) / 2, (o->s[i] + 1) / 2};
      double rr = 2 * lam[fa[f]] - 1, ss = 2 * lam[fb[f]] - 1;
      int best = -1;
      double bd = 1e300;
      for (int j = 0; j < Np; ++j) {
        double d = std::hypot(o->r[j] - rr, o->s[j] - ss);
        if (d < bd) { bd = d; best = j; }
      }
      if (bd > 1e-10) { *err = "node set not rotation symmetric"; return nullptr; }
      o->perm[f * Np + i] = best;
    }
  // reconstruction system: A1[m][n] = int_I phi_n psi_m, A2[m][n] = int_I phi_n(-r,-s) psi_m
  std::vector<double> gx, gw;
  gauss_legendre((3 * N + 2) / 2 + 2, gx, gw);
  Mat A((size_t)2 * Np * Mp, 0.0);
  std::vector<double> ps(Np);
  for (size_t qa = 0; qa < gx.size(); ++qa)
    for (size_t qb = 0; qb < gx.size(); ++qb) {
      double a = gx[qa], b = gx[qb];
      double rq = (1 + a) * (1 - b) / 2 - 1, sq = b, w = gw[qa] * gw[qb] * (1 - b) / 2;
      simplex_basis(N, rq, sq, ps.data(), nullptr, nullptr);
      for (int m = 0; m < Np; ++m)
        for (int ia = 0; ia <= N; ++ia)
          for (int ib = 0; ib <= N; ++ib) {
            int n = ia * (N + 1) + ib;
            A[(size_t)m * Mp + n] += w * ps[m] * legn(ia, rq) * legn(ib, sq);
            A[(size_t)(Np + m) * Mp + n] += w * ps[m] * legn(ia, -rq) * legn(ib, -sq);
          }
    }
  if (!pinv_qr(A, 2 * Np, Mp, o->Apinv, o->A_cond) || o->A_cond < 1e-10) {
    *err = "reconstruction system rank deficient";
    return nullptr;
  }
  // gradient of the tensor basis at the diagonal nodes (R,S) = (-t, t)
  Mat DR((size_t)Nfp * Mp), DS((size_t)Nfp * Mp);
  for (int i = 0; i < Nfp; ++i) {
    double R = -t[i], S = t[i];
    for (int ia = 0; ia <= N; ++ia)
      for (int ib = 0; ib <= N; ++ib) {
        int n = ia * (N + 1) + ib;
        DR[(size_t)i * Mp + n] = dlegn(ia, R) * legn(ib, S);
        DS[(size_t)i * Mp + n] = legn(ia, R) * dlegn(ib, S);
      }
  }
  Mat QR = matmul(DR, o->Apinv, Nfp, Mp, 2 * Np), QS = matmul(DS, o->Apinv, Nfp, Mp, 2 * Np);
  for (int k = 0; k < 2; ++k) {
    Mat qr((size_t)Nfp * Np), qs((size_t)Nfp * Np);
    for (int i = 0; i < Nfp; ++i)
      for (int j = 0; j < Np; ++j) {
        qr[(size_t)i * Np + j] = QR[(size_t)i * 2 * Np + k * Np + j];
        qs[(size_t)i * Np + j] = QS[(size_t)i * 2 * Np + k * Np + j];
      }
    o->QRV[k] = matmul(qr, o->Vinv, Nfp, Np, Np);
    o->QSV[k] = matmul(qs, o->Vinv, Nfp, Np, Np);
  }
  // Algorithm 1 factors: Y^rho_j = s_j Phi_diag A+_j (Vinv D_rho V) A_j, then Y A+_k Vinv
  {
    Mat Phi((size_t)Nfp * Mp);
    for (int i = 0; i < Nfp; ++i)
      for (int ia = 0; ia <= N; ++ia)
        for (int ib = 0; ib <= N; ++ib) Phi[(size_t)i * Mp + ia * (N + 1) + ib] = legn(ia, -t[i]) * legn(ib, t[i]);
    Mat DrM = matmul(matmul(o->Vinv, o->Dr, Np, Np, Np), o->V, Np, Np, Np);
    Mat DsM = matmul(matmul(o->Vinv, o->Ds, Np, Np, Np), o->V, Np, Np, Np);
    Mat Ap[2], Ak[2];
    for (int k = 0; k < 2; ++k) {
      Ap[k].resize((size_t)Mp * Np);
      Ak[k].resize((size_t)Np * Mp);
      for (int a = 0; a < Mp; ++a)
        for (int j = 0; j < Np; ++j) Ap[k][(size_t)a * Np + j] = o->Apinv[(size_t)a * 2 * Np + k * Np + j];
      for (int j = 0; j < Np; ++j)
        for (int a = 0; a < Mp; ++a) Ak[k][(size_t)j * Mp + a] = A[(size_t)(k * Np + j) * Mp + a];
    }
    for (int j = 0; j < 2; ++j) {
      const double sj = j == 0 ? 1.0 : -1.0;
      Mat PA = matmul(Phi, Ap[j], Nfp, Mp, Np);
      o->RVV[j] = matmul(PA, o->Vinv, Nfp, Np, Np);
      Mat DrVA = matmul(matmul(o->Dr, o->V, Np, Np, Np), Ak[j], Np, Np, Mp);
      Mat DsVA = matmul(matmul(o->Ds, o->V, Np, Np, Np), Ak[j], Np, Np, Mp);
      for (int k = 0; k < 2; ++k) {
        o->GR[j][k] = matmul(matmul(DrVA, Ap[k], Np, Mp, Np), o->Vinv, Np, Np, Np);
        o->GS[j][k] = matmul(matmul(DsVA, Ap[k], Np, Mp, Np), o->Vinv, Np, Np, Np);
      }
      Mat YR = matmul(matmul(PA, DrM, Nfp, Np, Np), Ak[j], Nfp, Np, Mp);
      Mat YS = matmul(matmul(PA, DsM, Nfp, Np, Np), Ak[j], Nfp, Np, Mp);
      for (auto& y : YR) y *= sj;
      for (auto& y : YS) y *= sj;
      for (int k = 0; k < 2; ++k) {
        o->ZR[j][k] = matmul(matmul(YR, Ap[k], Nfp, Mp, Np), o->Vinv, Nfp, Np, Np);
        o->ZS[j][k] = matmul(matmul(YS, Ap[k], Nfp, Mp, Np), o->Vinv, Nfp, Np, Np);
      }
    }
  }
  // reconstruction of the constant 1 on one side (0 on the other), evaluated on the diagonal
  {
    Mat ones(Np, 1.0);
    Mat chat = matmul(o->Vinv, ones, Np, Np, 1);   // projection of a constant is that constant
    Mat Phi((size_t)Nfp * Mp);
    for (int i = 0; i < Nfp; ++i)
      for (int ia = 0; ia <= N; ++ia)
        for (int ib = 0; ib <= N; ++ib) Phi[(size_t)i * Mp + ia * (N + 1) + ib] = legn(ia, -t[i]) * legn(ib, t[i]);
    Mat PA = matmul(Phi, o->Apinv, Nfp, Mp, 2 * Np);
    for (int k = 0; k < 2; ++k) {
      o->dvec[k].assign(Nfp, 0.0);
      for (int i = 0; i < Nfp; ++i)
        for (int m = 0; m < Np; ++m) o->dvec[k][i] += PA[(size_t)i * 2 * Np + k * Np + m] * chat[m];
    }
  }
  // GEMM form: C_m[n][j] = int_T psi_j(A_n(alpha, beta)) psi_m(alpha, beta), exact with a
  // collapsed Gauss rule (the integrand has degree <= 2N), A_n the affine image of node n.
  {
    std::vector<double> qx, qw;
    gauss_legendre(N + 3, qx, qw);
    Mat C((size_t)Np * Np * Np, 0.0);   // [m][n][j]
    std::vector<double> pm(Np), pj(Np);
    for (size_t qa = 0; qa < qx.size(); ++qa)
      for (size_t qb = 0; qb < qx.size(); ++qb) {
        const double a = qx[qa], b = qx[qb];
        const double al = (1 + a) * (1 - b) / 2 - 1, be = b, w = qw[qa] * qw[qb] * (1 - b) / 2;
        simplex_basis(N, al, be, pm.data(), nullptr, nullptr);
        for (int n = 0; n < Np; ++n) {
          const double rn = o->r[n], sn = o->s[n];
          const double Ar = -(rn + sn) / 2 * al + (rn + 1) / 2 - (sn + 1) / 2;
          const double As = -(rn + sn) / 2 * be - (rn + 1) / 2 + (sn + 1) / 2;
          simplex_basis(N, Ar, As, pj.data(), nullptr, nullptr);
          for (int m = 0; m < Np; ++m)
            for (int j = 0; j < Np; ++j) C[((size_t)m * Np + n) * Np + j] += w * pm[m] * pj[j];
        }
      }
    for (int k = 0; k < 2; ++k) {
      o->X[k].assign((size_t)Np * Nfp * 2 * Np, 0.0);
      for (int m = 0; m < Np; ++m) {
        Mat Cm(C.begin() + (size_t)m * Np * Np, C.begin() + (size_t)(m + 1) * Np * Np);
        Mat CV = matmul(Cm, o->Vinv, Np, Np, Np);
        Mat XR = matmul(o->QRV[k], CV, Nfp, Np, Np), XS = matmul(o->QSV[k], CV, Nfp, Np, Np);
        for (int i = 0; i < Nfp; ++i)
          for (int l = 0; l < Np; ++l) {
            o->X[k][(((size_t)m * Nfp + i) * 2 + 0) * Np + l] = XR[(size_t)i * Np + l];
            o->X[k][(((size_t)m * Nfp + i) * 2 + 1) * Np + l] = XS[(size_t)i * Np + l];
          }
      }
    }
    // the shared face in rotated order: the same nodes for every face f
    o->hyp.assign(Nfp, -1);
    for (int f = 0; f < 3; ++f)
      for (int q = 0; q < Nfp; ++q) {
        const int l = o->perm[f * Np + o->Fmask[f * Nfp + q]];
        if (f == 0) o->hyp[q] = l;
        else if (o->hyp[q] != l) { *err = "rotated face nodes differ between faces"; return nullptr; }
      }
  }
  return o;
}

std::mutex g_mu;
std::unique_ptr<RefOps> g_ops[kMaxN + 1];

}  // namespace

// psi_{ij}(r,s) = sqrt(2) P_i(a) P_j^{(2i+1,0)}(b) (1-b)^i, a = 2(1+r)/(1-s) - 1, b = s;
// gradients by the chain rule written so that no division by (1-s) remains.
void simplex_basis(int N, double r, double s, double* psi, double* dr, double* ds) {
  double a = (std::fabs(1 - s) > 1e-14) ? 2 * (1 + r) / (1 - s) - 1 : -1.0;
  double b = s;
  int m = 0;
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N - i; ++j, ++m) {
      double f = jacobi(a, 0, 0, i), df = jacobi_deriv(a, 0, 0, i);
      double g = jacobi(b, 2 * i + 1, 0, j), dg = jacobi_deriv(b, 2 * i + 1, 0, j);
      double omb_i = std::pow(1 - b, i);
      psi[m] = std::sqrt(2.0) * f * g * omb_i;
      if (dr) {
        double omb_im1 = (i > 0) ? std::pow(1 - b, i - 1) : 0.0;
        dr[m] = (i > 0) ? std::sqrt(2.0) * 2 * df * g * omb_im1 : 0.0;
        ds[m] = std::sqrt(2.0) * ((i > 0 ? df * (1 + a) * g * omb_im1 : 0.0) + f * dg * omb_i -
                                  (i > 0 ? i * f * g * omb_im1 : 0.0));
      }
    }
}

void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w) { gauss_legendre(n, x, w); }

const RefOps* get_refops(int N, const char** err) {
  static const char* kRange = "order N must be in 1..6";
  if (N < 1 || N > kMaxN) { if (err) *err = kRange; return nullptr; }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ops[N]) {
    const char* e = "";
    g_ops[N] = build(N, &e);
    if (!g_ops[N]) { if (err) *err = e; return nullptr; }
  }
  return g_ops[N].get();
}

}  // namespace rdg
