// FP64 setup kernels: element metric terms and, per edge, the enclosed parallelogram and the
// folded flux operator W_e (Sec. 4.2-4.5, Algorithm aRDG, Algorithm 2).
#include <cuda_runtime.h>

#include <cmath>

#include "internal.h"

namespace rdg {

// Reference-constant layout for order N (all doubles):
//   r[Np] s[Np] Vinv[Np][Np] QRV0 QSV0 QRV1 QSV1 ([Nfp][Np] each) perminv[3][Np] Fmask[3][Nfp]
//   dvec[2][Nfp]
std::vector<double> pack_setup_refs(const RefOps& o) {
  const int Np = o.Np, Nfp = o.Nfp;
  std::vector<double> v;
  v.insert(v.end(), o.r.begin(), o.r.end());
  v.insert(v.end(), o.s.begin(), o.s.end());
  v.insert(v.end(), o.Vinv.begin(), o.Vinv.end());
  for (int k = 0; k < 2; ++k) {
    v.insert(v.end(), o.QRV[k].begin(), o.QRV[k].end());
    v.insert(v.end(), o.QSV[k].begin(), o.QSV[k].end());
  }
  std::vector<double> pinv(3 * Np);
  for (int f = 0; f < 3; ++f)
    for (int i = 0; i < Np; ++i) pinv[f * Np + o.perm[f * Np + i]] = i;
  v.insert(v.end(), pinv.begin(), pinv.end());
  for (int x : o.Fmask) v.push_back(x);
  (void)Nfp;
  for (int k = 0; k < 2; ++k) v.insert(v.end(), o.dvec[k].begin(), o.dvec[k].end());
  return v;
}

namespace {

struct D2 {
  double x, y;
};
__device__ __forceinline__ D2 mk(double x, double y) { return D2{x, y}; }
__device__ __forceinline__ D2 operator+(D2 a, D2 b) { return mk(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ D2 operator-(D2 a, D2 b) { return mk(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ D2 operator*(double s, D2 a) { return mk(s * a.x, s * a.y); }
__device__ __forceinline__ double cross(D2 a, D2 b) { return a.x * b.y - a.y * b.x; }

// barycentric weights of the vertices b, c of triangle (a, b, c) at p
__device__ void bary(D2 p, D2 a, D2 b, D2 c, double& l2, double& l3) {
  D2 u = b - a, v = c - a, w = p - a;
  double det = cross(u, v);
  l2 = cross(w, v) / det;
  l3 = cross(u, w) / det;
}
__device__ bool inside(D2 p, D2 a, D2 b, D2 c) {
  double l2, l3;
  bary(p, a, b, c, l2, l3);
  const double tol = -1e-12;
  return l2 >= tol && l3 >= tol && (1.0 - l2 - l3) >= tol;
}
// intersection of the lines a0 + t (a1 - a0) and b0 + u (b1 - b0); ok = false if parallel
__device__ D2 cross_lines(D2 a0, D2 a1, D2 b0, D2 b1, bool& ok) {
  D2 da = a1 - a0, db = b1 - b0;
  double det = cross(da, db);
  ok = fabs(det) > 1e-300;
  double t = ok ? cross(b0 - a0, db) / det : 0.0;
  return a0 + t * da;
}

// Apex p1 of the maximum-area parallelogram with diagonal e1e2 inside T1 = (e1,e2,q1) and
// T2 = (e2,e1,q2): the highest point of T1 n (2c - T2).  That convex set's vertices are the
// base points, an apex lying in the other triangle, or a crossing of two slanted edges.
__device__ D2 parallelogram_apex(D2 e1, D2 e2, D2 q1, D2 q2) {
  const D2 c2 = e1 + e2;
  const D2 q2r = c2 - q2;
  const D2 d = e2 - e1;
  D2 best = e1;
  double hb = 0.0;
  auto consider = [&](D2 p) {
    if (inside(p, e1, e2, q1) && inside(p, e1, e2, q2r)) {
      double h = cross(d, p - e1);
      if (h > hb) { hb = h; best = p; }
    }
  };
  consider(q1);
  consider(q2r);
  bool ok;
  D2 x1 = cross_lines(e1, q1, e2, q2r, ok);
  if (ok) consider(x1);
  D2 x2 = cross_lines(e2, q1, e1, q2r, ok);
  if (ok) consider(x2);
  return best;
}

// (r, s) of p in the frame putting va at (1,-1), vb at (-1,1), vc at (-1,-1)
__device__ void frame_coords(D2 va, D2 vb, D2 vc, D2 p, double& r, double& s) {
  D2 a = 0.5 * (va - vc), b = 0.5 * (vb - vc), w = p - 0.5 * (va + vb);
  double det = cross(a, b);
  r = cross(w, b) / det;
  s = cross(a, w) / det;
}

// orthonormal Jacobi P_0..P_n^{(alpha,0)} at x
__device__ void jacobi_a0(double x, double al, int n, double* P) {
  const double g0 = pow(2.0, al + 1) / (al + 1);
  P[0] = 1.0 / sqrt(g0);
  if (n == 0) return;
  const double g1 = (al + 1) / (al + 3) * g0;
  P[1] = ((al + 2) * x / 2 + al / 2) / sqrt(g1);
  double aold = 2.0 / (2 + al) * sqrt((al + 1) / (al + 3));
  for (int i = 1; i < n; ++i) {
    const double h1 = 2 * i + al;
    const double anew = 2.0 / (h1 + 2) * sqrt((i + 1) * (i + 1 + al) * (i + 1 + al) * (i + 1) / (h1 + 1) / (h1 + 3));
    const double bnew = -(al * al) / h1 / (h1 + 2);
    P[i + 1] = (-aold * P[i - 1] + (x - bnew) * P[i]) / anew;
    aold = anew;
  }
}

template <int N>
__device__ void simplex_basis_dev(double r, double s, double* psi) {
  const double a = (fabs(1 - s) > 1e-14) ? 2 * (1 + r) / (1 - s) - 1 : -1.0;
  const double b = s;
  double Pa[N + 1], Pb[N + 1];
  jacobi_a0(a, 0.0, N, Pa);
  int m = 0;
  double omb = 1.0;
  for (int i = 0; i <= N; ++i) {
    jacobi_a0(b, 2 * i + 1, N - i, Pb);
    for (int j = 0; j <= N - i; ++j) psi[m++] = 1.4142135623730951 * Pa[i] * Pb[j] * omb;
    omb *= (1 - b);
  }
}

constexpr int kSetupWarps = 4;

template <int N>
__global__ void __launch_bounds__(32 * kSetupWarps) edge_setup_kernel(EdgeSetupIn in, void* Wt, int elem_bytes,
                                                                        double* Wd) {
  constexpr int NP = np_of(N), NFP = nfp_of(N), NW = NFP * 2 * NP;
  __shared__ double sVp[kSetupWarps][NP * NP];
  __shared__ double sB[kSetupWarps][NFP * NP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * kSetupWarps + warp;
  if (e >= in.E) return;   // whole warp leaves together; only __syncwarp is used below
  const double* R = in.refs;
  const double *rr = R, *ss = R + NP, *Vinv = R + 2 * NP;
  const double* QV = Vinv + NP * NP;  // QRV0 QSV0 QRV1 QSV1
  const double* perminv = QV + 4 * NFP * NP;
  const double* fmask = perminv + 3 * NP;
  const double* dvec = fmask + 3 * NFP;

  const int fa[3] = {0, 1, 2}, fb[3] = {1, 2, 0}, fc[3] = {2, 0, 1};
  const int k1 = in.k1[e], f1 = in.f1[e];
  int k2 = in.k2[e], f2 = in.f2[e];
  const double* x1 = in.xy + (int64_t)k1 * 6;
  const D2 e1 = mk(x1[2 * fa[f1]], x1[2 * fa[f1] + 1]);
  const D2 e2 = mk(x1[2 * fb[f1]], x1[2 * fb[f1] + 1]);
  const D2 q1 = mk(x1[2 * fc[f1]], x1[2 * fc[f1] + 1]);
  D2 q2;
  double D2v;
  if (k2 >= 0) {
    const double* x2 = in.xy + (int64_t)k2 * 6;
    q2 = mk(x2[2 * fc[f2]] + in.shift[2 * e], x2[2 * fc[f2] + 1] + in.shift[2 * e + 1]);
    D2v = in.D[k2];
  } else {
    q2 = (e1 + e2) - q1;   // ghost: point reflection of element k1 about the edge midpoint
    f2 = 1;                // the ghost's hypotenuse is the shared edge
    D2v = in.D[k1];
  }
  const double D1v = in.D[k1];
  const D2 p1 = parallelogram_apex(e1, e2, q1, q2);
  const D2 p2 = (e1 + e2) - p1;
  double al[2], be[2];
  frame_coords(e1, e2, q1, p1, al[0], be[0]);
  frame_coords(e2, e1, q2, p2, al[1], be[1]);
  const D2 d = e2 - e1;
  const double len = sqrt(d.x * d.x + d.y * d.y);
  const D2 n1 = mk(d.y / len, -d.x / len);
  const double Jf = 0.5 * len;
  const D2 xR = 0.5 * (e1 - p1), xS = 0.5 * (e2 - p1);
  const double Jp = cross(xR, xS);
  const double Rx = xS.y / Jp, Ry = -xS.x / Jp, Sx = -xR.y / Jp, Sy = xR.x / Jp;
  const double kR = n1.x * Rx + n1.y * Ry, kS = n1.x * Sx + n1.y * Sy;
  const double vn = n1.x * in.vx + n1.y * in.vy;
  const int ff[2] = {f1, f2};
  const int64_t tile = e >> 5, le = e & 31;
  const int VW = 16 / elem_bytes;
  const int QW = (NW + VW - 1) / VW;

  for (int side = 0; side < 2; ++side) {
    if (lane < NP) {
      const double rn = rr[lane], sn = ss[lane];
      const double Ar = -(rn + sn) / 2 * al[side] + (rn + 1) / 2 - (sn + 1) / 2;
      const double As = -(rn + sn) / 2 * be[side] - (rn + 1) / 2 + (sn + 1) / 2;
      simplex_basis_dev<N>(Ar, As, &sVp[warp][lane * NP]);
    }
    __syncwarp();
    if (lane < NP) {
      const double* QRV = QV + (2 * side) * NFP * NP;
      const double* QSV = QV + (2 * side + 1) * NFP * NP;
      for (int i = 0; i < NFP; ++i) {
        double acc = 0.0;
        for (int n = 0; n < NP; ++n) acc += (kR * QRV[i * NP + n] + kS * QSV[i * NP + n]) * sVp[warp][n * NP + lane];
        sB[warp][i * NP + lane] = acc;
      }
    }
    __syncwarp();
    if (lane < NP) {
      const int f = ff[side];
      const int col = (int)perminv[f * NP + lane];
      for (int i = 0; i < NFP; ++i) {
        double c = 0.0;
        for (int j = 0; j < NP; ++j) c += sB[warp][i * NP + j] * Vinv[j * NP + lane];
        const double Dt = in.iface == RDG_IFACE_HARMONIC ? 2.0 * D1v * D2v / (D1v + D2v)
                                                         : D1v * dvec[i] + D2v * dvec[NFP + i];
        double w = -Jf * Dt * c;
        if (side == 0 && vn >= 0 && col == (int)fmask[f1 * NFP + i]) w += Jf * vn;
        if (side == 1 && vn < 0 && col == (int)fmask[f2 * NFP + (NFP - 1 - i)]) w += Jf * vn;
        const int idx = i * 2 * NP + side * NP + col;
        const int64_t off = ((tile * QW + idx / VW) * kTile + le) * VW + (idx % VW);
        if (Wt) {
          if (elem_bytes == 4) static_cast<float*>(Wt)[off] = (float)w;
          else static_cast<double*>(Wt)[off] = w;
        }
        if (Wd) Wd[e * NW + idx] = w;
      }
    }
    __syncwarp();
  }
}

__global__ void elem_setup_kernel(int64_t K, const double* xy, const double* D, double vx, double vy, void* geo,
                                  int elem_bytes) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double* v = xy + k * 6;
  const double xr = 0.5 * (v[2] - v[0]), yr = 0.5 * (v[3] - v[1]);
  const double xs = 0.5 * (v[4] - v[0]), ys = 0.5 * (v[5] - v[1]);
  const double J = xr * ys - xs * yr;
  const double rx = ys / J, ry = -xs / J, sx = -yr / J, sy = xr / J;
  const double Dk = D[k];
  const double g[6] = {rx * vx + ry * vy, sx * vx + sy * vy, Dk * (rx * rx + ry * ry), Dk * (rx * sx + ry * sy),
                       Dk * (sx * sx + sy * sy), 1.0 / J};
  for (int c = 0; c < 6; ++c) {
    if (elem_bytes == 4) static_cast<float*>(geo)[c * K + k] = (float)g[c];
    else static_cast<double*>(geo)[c * K + k] = g[c];
  }
}

__global__ void advance_kernel(TimeState* ts, long long by) { ts->n += by; }
__global__ void set_time_kernel(TimeState* ts, double t0) {
  ts->t0 = t0;
  ts->n = 0;
}

}  // namespace

int setup_edges(int N, const EdgeSetupIn& in, void* W_tiled, int elem_bytes, double* W_dense, cudaStream_t s) {
  if (in.E == 0) return RDG_OK;
  const unsigned grid = (unsigned)((in.E + kSetupWarps - 1) / kSetupWarps);
  switch (N) {
    case 1: edge_setup_kernel<1><<<grid, 32 * kSetupWarps, 0, s>>>(in, W_tiled, elem_bytes, W_dense); break;
    case 2: edge_setup_kernel<2><<<grid, 32 * kSetupWarps, 0, s>>>(in, W_tiled, elem_bytes, W_dense); break;
    case 3: edge_setup_kernel<3><<<grid, 32 * kSetupWarps, 0, s>>>(in, W_tiled, elem_bytes, W_dense); break;
    case 4: edge_setup_kernel<4><<<grid, 32 * kSetupWarps, 0, s>>>(in, W_tiled, elem_bytes, W_dense); break;
    case 5: edge_setup_kernel<5><<<grid, 32 * kSetupWarps, 0, s>>>(in, W_tiled, elem_bytes, W_dense); break;
    case 6: edge_setup_kernel<6><<<grid, 32 * kSetupWarps, 0, s>>>(in, W_tiled, elem_bytes, W_dense); break;
    default: return RDG_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

int setup_elements(int64_t K, const double* xy, const double* D, double vx, double vy, void* geo, int elem_bytes,
                   cudaStream_t s) {
  if (K == 0) return RDG_OK;
  elem_setup_kernel<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(K, xy, D, vx, vy, geo, elem_bytes);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

int set_time(TimeState* ts, double t0, cudaStream_t s) {
  set_time_kernel<<<1, 1, 0, s>>>(ts, t0);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

int advance_time(TimeState* ts, long long by, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(ts, by);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

}  // namespace rdg
