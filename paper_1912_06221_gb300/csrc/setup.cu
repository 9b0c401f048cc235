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
  // Recurrence constants of the orthonormal Jacobi polynomials P_n^{(al,0)} (the collapsed
  // coordinate factors of the simplex basis) for al = 0 and al = 2i+1, i = 0..N, so the
  // device evaluates the basis with multiply-adds only (FP64 square roots and divisions are
  // slow on this part).  Per al, 3N values: c0 = 1/sqrt(g0), P_1 = c1a x + c1b, and for
  // n = 1..N-1 (A_n, B_n, C_n) with P_{n+1} = (x - B_n) A_n P_n - C_n P_{n-1}.
  const int N = Nfp - 1;
  for (int ai = 0; ai <= N + 1; ++ai) {
    const double al = ai == 0 ? 0.0 : 2.0 * (ai - 1) + 1.0;
    const double g0 = std::pow(2.0, al + 1) / (al + 1);
    const double g1 = (al + 1) / (al + 3) * g0;
    v.push_back(1.0 / std::sqrt(g0));
    v.push_back((al + 2) / 2 / std::sqrt(g1));
    v.push_back(al / 2 / std::sqrt(g1));
    double aold = 2.0 / (2 + al) * std::sqrt((al + 1) / (al + 3));
    for (int n = 1; n < N; ++n) {
      const double h1 = 2 * n + al;
      const double anew =
          2.0 / (h1 + 2) * std::sqrt((n + 1) * (n + 1 + al) * (n + 1 + al) * (n + 1) / (h1 + 1) / (h1 + 3));
      const double bnew = -(al * al) / h1 / (h1 + 2);
      v.push_back(1.0 / anew);
      v.push_back(bnew);
      v.push_back(aold / anew);
      aold = anew;
    }
  }
  // Algorithm 1 factors per input side k: ZR[0][k], ZS[0][k] (weight D1), ZR[1][k], ZS[1][k] (D2)
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j) {
      v.insert(v.end(), o.ZR[j][k].begin(), o.ZR[j][k].end());
      v.insert(v.end(), o.ZS[j][k].begin(), o.ZS[j][k].end());
    }
  (void)Np;
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

// Orthonormal Jacobi P_0..P_n^{(al,0)} at x from the recurrence constants t (3N values, the
// layout pack_setup_refs writes).
__device__ __forceinline__ void jacobi_tab(double x, const double* t, int n, double* P) {
  P[0] = t[0];
  if (n == 0) return;
  P[1] = fma(t[1], x, t[2]);
  for (int k = 1; k < n; ++k) P[k + 1] = (x - t[3 * k + 1]) * t[3 * k] * P[k] - t[3 * k + 2] * P[k - 1];
}

// Orthonormal simplex basis psi_m(r, s), m = (i, j) with i + j <= N in i-major order: the
// collapsed coordinates a = 2(1+r)/(1-s) - 1, b = s and psi = sqrt(2) P_i(a) P_j^{(2i+1,0)}(b)
// (1-b)^i.  jac holds the constants for al = 0 then al = 2i+1, 3N values each.
template <int N>
__device__ void simplex_basis_tab(double r, double s, const double* jac, double* psi) {
  const double a = (fabs(1 - s) > 1e-14) ? 2 * (1 + r) / (1 - s) - 1 : -1.0;
  const double b = s;
  double Pa[N + 1], Pb[N + 1];
  jacobi_tab(a, jac, N, Pa);
  int m = 0;
  double omb = 1.0;
#pragma unroll
  for (int i = 0; i <= N; ++i) {
    jacobi_tab(b, jac + 3 * N * (i + 1), N - i, Pb);
    for (int j = 0; j <= N - i; ++j) psi[m++] = 1.4142135623730951 * Pa[i] * Pb[j] * omb;
    omb *= (1 - b);
  }
}

// Warps (one edge each) per block of the set-up kernel: the reference constants are staged
// once per block in shared memory, plus NP^2 + 2 Nfp NP doubles per warp (under 48 KB).
template <int N>
__host__ __device__ constexpr int setup_warps() {
  return N >= 6 ? 2 : 4;
}

template <int N>
__host__ __device__ constexpr int setup_ref_count() {
  constexpr int NP = np_of(N), NFP = nfp_of(N);
  return 2 * NP + NP * NP + 4 * NFP * NP + 3 * NP + 3 * NFP + 2 * NFP + 3 * N * (N + 2) + 8 * NFP * NP;
}

// One warp per edge: the parallelogram apex, the two rotated frames and the metric (lane
// uniform), then per side the basis at the side's nodes mapped into the parallelogram frame
// (one lane per node) and the two small products (kR QR + kS QS) V_p and (.) V^{-1} spread
// over all 32 lanes.
template <int N>
__global__ void __launch_bounds__(32 * setup_warps<N>()) edge_setup_kernel(EdgeSetupIn in, void* Wt, int elem_bytes,
                                                                            double* Wd, float* Pt) {
  constexpr int NP = np_of(N), NFP = nfp_of(N), NW = NFP * 2 * NP, WARPS = setup_warps<N>();
  constexpr int RT = setup_ref_count<N>();
  __shared__ double sR[RT];
  // the basis at both sides' mapped nodes in one pass of the warp where 2 Np lanes fit (N <= 4),
  // so the FP64 pipe (the set-up's bound) is not half idle for the table; one side at a time above
  constexpr bool BOTH = 2 * NP <= 32;
  __shared__ double sVp[WARPS][(BOTH ? 2 : 1) * NP * NP];
  __shared__ double sK[WARPS][NFP * NP];
  __shared__ double sB[WARPS][NFP * NP];
  __shared__ double sD[WARPS][2 * NP + NFP];   // nodal D: d_j at side j's sub-triangle nodes, then D~_i
  for (int i = threadIdx.x; i < RT; i += blockDim.x) sR[i] = in.refs[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * WARPS + warp;
  if (e >= in.E) return;   // whole warp leaves together; only __syncwarp is used below
  const double *rr = sR, *ss = sR + NP, *Vinv = sR + 2 * NP;
  const double* QV = Vinv + NP * NP;  // QRV0 QSV0 QRV1 QSV1
  const double* perminv = QV + 4 * NFP * NP;
  const double* fmask = perminv + 3 * NP;
  const double* dvec = fmask + 3 * NFP;
  const double* jac = dvec + 2 * NFP;
  const double* zq = jac + 3 * N * (N + 2);   // Algorithm 1 factors, 4 Nfp x Np per input side

  const int fa[3] = {0, 1, 2}, fb[3] = {1, 2, 0}, fc[3] = {2, 0, 1};
  const int k1 = in.k1[e], f1 = in.f1[e];
  int k2 = in.k2[e], f2 = in.f2[e];
  const double* x1 = in.xy + (int64_t)k1 * 6;
  const D2 e1 = mk(x1[2 * fa[f1]], x1[2 * fa[f1] + 1]);
  const D2 e2 = mk(x1[2 * fb[f1]], x1[2 * fb[f1] + 1]);
  const D2 q1 = mk(x1[2 * fc[f1]], x1[2 * fc[f1] + 1]);
  D2 q2;
  double D2v, D2y;
  const bool aniso = in.Dy != nullptr;   // diagonal tensor (Dx, Dy); D holds Dx
  if (k2 >= 0) {
    const double* x2 = in.xy + (int64_t)k2 * 6;
    q2 = mk(x2[2 * fc[f2]] + in.shift[2 * e], x2[2 * fc[f2] + 1] + in.shift[2 * e + 1]);
    D2v = in.D[k2];
    D2y = aniso ? in.Dy[k2] : D2v;
  } else {
    q2 = (e1 + e2) - q1;   // ghost: point reflection of element k1 about the edge midpoint
    f2 = 1;                // the ghost's hypotenuse is the shared edge
    D2v = in.D[k1];
    D2y = aniso ? in.Dy[k1] : D2v;
  }
  const double D1v = in.D[k1];
  const double D1y = aniso ? in.Dy[k1] : D1v;
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
  const bool nodal = in.Dn != nullptr;
  if (nodal) {
    // D at each side's sub-triangle nodes: d_j = V_pj V_rf^{-1} D_j, the element's nodal D
    // (a ghost: its element's D at the reflected points) in the rotated order of the side's face
    double* dn = sB[warp];                  // scratch: the side's nodal D, then its modal values
    for (int side = 0; side < 2; ++side) {
      const int kk = side == 0 ? k1 : k2;
      if (kk >= 0) {
        if (lane < NP) dn[lane] = in.Dn[(int64_t)kk * NP + lane];
      } else {
        // a ghost's node (barycentric l1, l2, l3 on its vertices: reflected apex, e2, e1) is
        // the reflection of element k1's point with l1 at its apex, l2 at e1 and l3 at e2, so
        // the ghost's D there is k1's D at that point: k1's modal D, evaluated
        double modal = 0.0;
        if (lane < NP)
          for (int l = 0; l < NP; ++l) modal = fma(Vinv[lane * NP + l], in.Dn[(int64_t)k1 * NP + l], modal);
        if (lane < NP) dn[NP + lane] = modal;
        __syncwarp();
        double val = 0.0;
        if (lane < NP) {
          const double l1 = -(rr[lane] + ss[lane]) / 2, l2 = (rr[lane] + 1) / 2, l3 = (ss[lane] + 1) / 2;
          double L[3];
          L[fc[f1]] = l1;
          L[fa[f1]] = l2;
          L[fb[f1]] = l3;
          double ph[NP];
          simplex_basis_tab<N>(2 * L[1] - 1, 2 * L[2] - 1, jac, ph);
          for (int m = 0; m < NP; ++m) val = fma(ph[m], dn[NP + m], val);
        }
        __syncwarp();
        if (lane < NP) dn[lane] = val;
      }
      __syncwarp();
      // modal coefficients of the rotated nodal D, then values at the sub-triangle nodes
      const int f = ff[side];
      double mo = 0.0;
      if (lane < NP)
        for (int l = 0; l < NP; ++l) mo = fma(Vinv[lane * NP + l], dn[(int)perminv[f * NP + l]], mo);
      __syncwarp();
      if (lane < NP) dn[NP + lane] = mo;
      if (lane < NP) {
        const double rn = rr[lane], sn = ss[lane];
        const double Ar = -(rn + sn) / 2 * al[side] + (rn + 1) / 2 - (sn + 1) / 2;
        const double As = -(rn + sn) / 2 * be[side] - (rn + 1) / 2 + (sn + 1) / 2;
        simplex_basis_tab<N>(Ar, As, jac, &sVp[warp][lane * NP]);
      }
      __syncwarp();
      if (lane < NP) {
        double d = 0.0;
        for (int m = 0; m < NP; ++m) d = fma(sVp[warp][lane * NP + m], dn[NP + m], d);
        sD[warp][side * NP + lane] = d;
      }
      __syncwarp();
    }
    // edge coefficient per diagonal node: Algorithm 2 reconstructs D from both sides' nodal
    // data (D~ = sum_j RVV_j d_j); the harmonic rule takes the two traces at the face node
    if (lane < NFP) {
      const int i = lane;
      double dt;
      if (in.iface == RDG_IFACE_HARMONIC) {
        const double t1 = in.Dn[(int64_t)k1 * NP + (int)fmask[f1 * NFP + i]];
        // side 2's face node matching side 1's node i (its face runs the other way)
        const int col2 = (int)fmask[f2 * NFP + (NFP - 1 - i)];
        // (a ghost's D at that point is its element's at the mirrored face node)
        const double t2 = k2 >= 0 ? in.Dn[(int64_t)k2 * NP + col2]
                                  : in.Dn[(int64_t)k1 * NP + (int)fmask[f1 * NFP + (NFP - 1 - i)]];
        dt = 2.0 * t1 * t2 / (t1 + t2);
      } else {
        const double* RVV = in.nodal_refs;
        dt = 0.0;
        for (int j = 0; j < 2; ++j)
          for (int n = 0; n < NP; ++n) dt = fma(RVV[(j * NFP + i) * NP + n], sD[warp][j * NP + n], dt);
      }
      sD[warp][2 * NP + i] = dt;
    }
    __syncwarp();
  }
  const int VW = 16 / elem_bytes;
  const int QW = (NFP * (2 * NP - 1) + 1 + VW - 1) / VW;   // 16-byte words of the stored operator

  if (Pt) {
    // GEMM-form parameter record (FP32): psi_m(alpha_k, beta_k) of both sides, kappa_R,
    // kappa_S, -J_f D~_i and J_f (v.n1), tiled [edge/32][16-byte word][lane]
    constexpr int PW = 2 * NP + NFP + 3, PW4 = (PW + 3) / 4;
    auto put = [&](int j, double x) {
      Pt[(((tile * PW4 + j / 4) * kTile) + le) * 4 + (j % 4)] = (float)x;
    };
    if (lane < 2) {
      double ph[NP];
      simplex_basis_tab<N>(al[lane], be[lane], jac, ph);
      for (int m = 0; m < NP; ++m) put(lane * NP + m, ph[m]);
    } else if (lane == 2) {
      put(2 * NP, kR);
      put(2 * NP + 1, kS);
      for (int i = 0; i < NFP; ++i) {
        const double Dt = in.iface == RDG_IFACE_HARMONIC ? 2.0 * D1v * D2v / (D1v + D2v)
                                                         : D1v * dvec[i] + D2v * dvec[NFP + i];
        put(2 * NP + 2 + i, -Jf * Dt);
      }
      put(2 * NP + 2 + NFP, Jf * vn);
      for (int j = PW; j < 4 * PW4; ++j) put(j, 0.0);
    }
    if (!Wt && !Wd) return;
  }
  if constexpr (BOTH) {
    if (lane < 2 * NP) {
      const int sd = lane / NP, nd = lane % NP;
      const double rn = rr[nd], sn = ss[nd];
      const double Ar = -(rn + sn) / 2 * al[sd] + (rn + 1) / 2 - (sn + 1) / 2;
      const double As = -(rn + sn) / 2 * be[sd] - (rn + 1) / 2 + (sn + 1) / 2;
      simplex_basis_tab<N>(Ar, As, jac, &sVp[warp][sd * NP * NP + nd * NP]);
    }
    __syncwarp();
  }
  for (int side = 0; side < 2; ++side) {
    if (!BOTH && lane < NP) {
      const double rn = rr[lane], sn = ss[lane];
      const double Ar = -(rn + sn) / 2 * al[side] + (rn + 1) / 2 - (sn + 1) / 2;
      const double As = -(rn + sn) / 2 * be[side] - (rn + 1) / 2 + (sn + 1) / 2;
      simplex_basis_tab<N>(Ar, As, jac, &sVp[warp][lane * NP]);
    }
    const double* vp = &sVp[warp][BOTH ? side * NP * NP : 0];
    const double* QRV = QV + (2 * side) * NFP * NP;
    const double* QSV = QV + (2 * side + 1) * NFP * NP;
    if (in.iface == RDG_IFACE_ALG1 && nodal) {
      // Algorithm 1 with D at the sub-triangle nodes: sum_j s_j RVV_j diag(d_j)
      // (kappa_R GR[j][side] + kappa_S GS[j][side])
      const double* RVV = in.nodal_refs;
      const double* GRb = RVV + 2 * NFP * NP;
      const double* GSb = GRb + 4 * NP * NP;
      for (int t = lane; t < NFP * NP; t += 32) {
        const int i = t / NP, l = t % NP;
        double acc = 0.0;
        for (int j = 0; j < 2; ++j) {
          const double sj = j == 0 ? 1.0 : -1.0;
          const double* gr = GRb + (j * 2 + side) * NP * NP;
          const double* gs = GSb + (j * 2 + side) * NP * NP;
          for (int n = 0; n < NP; ++n)
            acc = fma(sj * RVV[(j * NFP + i) * NP + n] * sD[warp][j * NP + n], kR * gr[n * NP + l] + kS * gs[n * NP + l],
                      acc);
        }
        sK[warp][t] = acc;
      }
    } else if (in.iface == RDG_IFACE_ALG1 && aniso) {
      // Algorithm 1 with D = (Dx, Dy): sub-triangle j's product is (Dx^j u~_x, Dy^j u~_y), so its
      // R and S parts carry n_x Dx^j R_x + n_y Dy^j R_y and n_x Dx^j S_x + n_y Dy^j S_y
      const double* Z = zq + side * 4 * NFP * NP;
      const double aR1 = n1.x * D1v * Rx + n1.y * D1y * Ry, aS1 = n1.x * D1v * Sx + n1.y * D1y * Sy;
      const double aR2 = n1.x * D2v * Rx + n1.y * D2y * Ry, aS2 = n1.x * D2v * Sx + n1.y * D2y * Sy;
      for (int t = lane; t < NFP * NP; t += 32)
        sK[warp][t] = aR1 * Z[t] + aS1 * Z[NFP * NP + t] + aR2 * Z[2 * NFP * NP + t] + aS2 * Z[3 * NFP * NP + t];
    } else if (in.iface == RDG_IFACE_ALG1) {
      // Algorithm 1: D_1 (kR ZR[0] + kS ZS[0]) + D_2 (kR ZR[1] + kS ZS[1]) for this side
      const double* Z = zq + side * 4 * NFP * NP;
      for (int t = lane; t < NFP * NP; t += 32)
        sK[warp][t] = D1v * (kR * Z[t] + kS * Z[NFP * NP + t]) + D2v * (kR * Z[2 * NFP * NP + t] + kS * Z[3 * NFP * NP + t]);
    } else if (aniso) {
      // Algorithm 2 (or the harmonic rule) per component: n1 . (D~x u~_x, D~y u~_y) at diagonal
      // node i, i.e. row i carries n_x D~x_i R_x + n_y D~y_i R_y and the same with S
      for (int t = lane; t < NFP * NP; t += 32) {
        const int i = t / NP;
        const bool hm = in.iface == RDG_IFACE_HARMONIC;
        const double Dtx = hm ? 2.0 * D1v * D2v / (D1v + D2v) : D1v * dvec[i] + D2v * dvec[NFP + i];
        const double Dty = hm ? 2.0 * D1y * D2y / (D1y + D2y) : D1y * dvec[i] + D2y * dvec[NFP + i];
        sK[warp][t] = (n1.x * Dtx * Rx + n1.y * Dty * Ry) * QRV[t] + (n1.x * Dtx * Sx + n1.y * Dty * Sy) * QSV[t];
      }
    } else {
      for (int t = lane; t < NFP * NP; t += 32) sK[warp][t] = kR * QRV[t] + kS * QSV[t];
    }
    __syncwarp();
    for (int t = lane; t < NFP * NP; t += 32) {
      const int i = t / NP, j = t % NP;
      double acc = 0.0;
#pragma unroll 7
      for (int n = 0; n < NP; ++n) acc = fma(sK[warp][i * NP + n], vp[n * NP + j], acc);
      sB[warp][t] = acc;
    }
    __syncwarp();
    const int f = ff[side];
    for (int t = lane; t < NFP * NP; t += 32) {
      const int i = t / NP, l = t % NP;
      double c = 0.0;
#pragma unroll 7
      for (int j = 0; j < NP; ++j) c = fma(sB[warp][i * NP + j], Vinv[j * NP + l], c);
      const int col = (int)perminv[f * NP + l];
      const double Dt = (in.iface == RDG_IFACE_ALG1 || aniso) ? 1.0   // D inside the factors
                        : nodal                                   ? sD[warp][2 * NP + i]
                        : in.iface == RDG_IFACE_HARMONIC ? 2.0 * D1v * D2v / (D1v + D2v)
                                                         : D1v * dvec[i] + D2v * dvec[NFP + i];
      double w = -Jf * Dt * c;
      if (side == 0 && vn >= 0 && col == (int)fmask[f1 * NFP + i]) w += Jf * vn;
      if (side == 1 && vn < 0 && col == (int)fmask[f2 * NFP + (NFP - 1 - i)]) w += Jf * vn;
      const int idx = i * 2 * NP + side * NP + col;
      // Stored (difference) form: the flux kernels apply the operator to
      // (u_0, u_1 - u_0, ..., u_{2Np-1} - u_0), u_0 = side 1's first node value, so column 0
      // would hold the row sum of W.  The reconstruction reproduces constants and their
      // gradient vanishes, so that row sum is the upwind part alone, J_f (v.n1), the same for
      // every row: it is stored once, after the rows' other 2 Np - 1 columns, and the large
      // diffusive entries only ever multiply differences of nearby values.
      constexpr int RW = 2 * NP - 1;
      int sidx = -1;
      if (side == 0 && col == 0) {
        if (i == 0) sidx = NFP * RW;                           // the shared row sum
      } else {
        sidx = i * RW + (side == 0 ? col - 1 : NP - 1 + col);
      }
      if (Wt && sidx >= 0) {
        const double wt = sidx == NFP * RW ? Jf * vn : w;
        const int64_t off = ((tile * QW + sidx / VW) * kTile + le) * VW + (sidx % VW);
        if (elem_bytes == 4) static_cast<float*>(Wt)[off] = (float)wt;
        else static_cast<double*>(Wt)[off] = wt;
      }
      if (Wd) Wd[e * NW + idx] = w;
    }
    __syncwarp();
  }
}

__global__ void elem_setup_kernel(int64_t K, const double* xy, const double* D, const double* Dy, double vx, double vy,
                                  void* geo, int elem_bytes) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const double* v = xy + k * 6;
  const double xr = 0.5 * (v[2] - v[0]), yr = 0.5 * (v[3] - v[1]);
  const double xs = 0.5 * (v[4] - v[0]), ys = 0.5 * (v[5] - v[1]);
  const double J = xr * ys - xs * yr;
  const double rx = ys / J, ry = -xs / J, sx = -yr / J, sy = xr / J;
  // F_r = r . F, F_s = s . F with F = v u - (Dx u_x, Dy u_y): g_ab = Dx a_x b_x + Dy a_y b_y
  const double Dx = D ? D[k] : 1.0;   // null: D given at the nodes, the metric alone here
  double g[6] = {rx * vx + ry * vy, sx * vx + sy * vy, Dx * (rx * rx + ry * ry), Dx * (rx * sx + ry * sy),
                 Dx * (sx * sx + sy * sy), 1.0 / J};
  if (Dy) {
    const double Dyk = Dy[k];
    g[2] = Dx * rx * rx + Dyk * ry * ry;
    g[3] = Dx * rx * sx + Dyk * ry * sy;
    g[4] = Dx * sx * sx + Dyk * sy * sy;
  }
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

template <int N>
int launch_setup(const EdgeSetupIn& in, void* W_tiled, int elem_bytes, double* W_dense, float* P_tiled,
                 cudaStream_t s) {
  constexpr int W = setup_warps<N>();
  if (in.nrefs != setup_ref_count<N>()) return RDG_EINVAL;
  const unsigned grid = (unsigned)((in.E + W - 1) / W);
  edge_setup_kernel<N><<<grid, 32 * W, 0, s>>>(in, W_tiled, elem_bytes, W_dense, P_tiled);
  return cudaGetLastError() == cudaSuccess ? RDG_OK : RDG_ECUDA;
}

int setup_edges(int N, const EdgeSetupIn& in, void* W_tiled, int elem_bytes, double* W_dense, float* P_tiled,
                cudaStream_t s) {
  if (in.E == 0) return RDG_OK;
  switch (N) {
    case 1: return launch_setup<1>(in, W_tiled, elem_bytes, W_dense, P_tiled, s);
    case 2: return launch_setup<2>(in, W_tiled, elem_bytes, W_dense, P_tiled, s);
    case 3: return launch_setup<3>(in, W_tiled, elem_bytes, W_dense, P_tiled, s);
    case 4: return launch_setup<4>(in, W_tiled, elem_bytes, W_dense, P_tiled, s);
    case 5: return launch_setup<5>(in, W_tiled, elem_bytes, W_dense, P_tiled, s);
    case 6: return launch_setup<6>(in, W_tiled, elem_bytes, W_dense, P_tiled, s);
    default: return RDG_EINVAL;
  }
}

int setup_elements(int64_t K, const double* xy, const double* D, const double* Dy, double vx, double vy, void* geo,
                   int elem_bytes, cudaStream_t s) {
  if (K == 0) return RDG_OK;
  elem_setup_kernel<<<(unsigned)((K + 255) / 256), 256, 0, s>>>(K, xy, D, Dy, vx, vy, geo, elem_bytes);
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
