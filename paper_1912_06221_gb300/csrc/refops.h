// Host FP64 reference-element operators of the aRDG method, one set per order N = 1..6.
// All of these are constants of the reference triangle / logical square, computed once per
// order and copied to the device.
#pragma once
#include <vector>

#ifdef __CUDACC__
#define RDG_HD __host__ __device__
#else
#define RDG_HD
#endif

namespace rdg {

constexpr int kMaxN = 6;
RDG_HD constexpr int np_of(int N) { return (N + 1) * (N + 2) / 2; }
RDG_HD constexpr int nfp_of(int N) { return N + 1; }
RDG_HD constexpr int mp_of(int N) { return (N + 1) * (N + 1); }

struct RefOps {
  int N = 0, Np = 0, Nfp = 0, Mp = 0;
  std::vector<double> r, s;          // nodes [Np]
  std::vector<double> V, Vinv;       // Vandermonde (orthonormal basis) [Np][Np], row = node
  std::vector<double> M;             // mass matrix [Np][Np]
  std::vector<double> Dr, Ds;        // differentiation [Np][Np]
  std::vector<double> Wr, Ws;        // weak derivatives M^{-1} Dr^T M, M^{-1} Ds^T M
  std::vector<double> LIFT;          // [Np][3*Nfp]: column f*Nfp+q
  std::vector<int> Fmask;            // [3][Nfp] face nodes, counter-clockwise
  std::vector<int> perm;             // [3][Np]: rotated node i of face f sits at node perm[f][i]
  std::vector<double> Apinv;         // [Mp][2Np] pseudo-inverse of the reconstruction system
  double A_cond = 0;                 // smallest/largest |R_ii| of its QR factor
  // per side k = 0,1: (DR A+)_k Vinv and (DS A+)_k Vinv, [Nfp][Np] each
  std::vector<double> QRV[2], QSV[2];
  // Algorithm 2 for element-constant D: D~(diagonal node i) = D1 dvec[0][i] + D2 dvec[1][i],
  // the reconstruction of the two constants through the same least-squares operator
  std::vector<double> dvec[2];
  // Reference factors of the on-the-fly flux (the GEMM form of the edge operator).  The
  // projection V_p(alpha, beta) of side k is a polynomial of degree <= N in the apex
  // coordinates (the map A is affine in them), expanded in the orthonormal basis:
  // V_p = sum_m psi_m(alpha, beta) C_m.  Then the side's diffusive operator in the rotated
  // node order is  sum_rho kappa_rho sum_m psi_m(alpha, beta) X[k][m][i][rho][l]  with
  // X[k][m][.][rho][.] = Q^rho_k C_m Vinv (Q^R = QRV, Q^S = QSV), layout
  // [m][Nfp][2][Np] per side.
  std::vector<double> X[2];
  // Algorithm 1 (n . RDG(D_1 grad u~^1, D_2 grad u~^2), Separation = L2 projection onto the
  // sub-triangles): the edge gradient is sum_j D_j (kappa_R ZR[j][k] + kappa_S ZS[j][k]) u_k,rot
  // summed over input sides k, with ZR[j][k] = Y^R_j A+_k Vinv, Y^R_j = s_j Phi_diag A+_j
  // (Vinv Dr V) A_j (s_1 = 1, s_2 = -1 for side 2's reflected frame), [Nfp][Np] each.
  std::vector<double> ZR[2][2], ZS[2][2];
  // The same factors split where a nodal D enters (D given at the nodes, multiplied into the
  // sub-triangle's nodal gradient): ZR[j][k] = s_j RVV[j] diag(1) GR[j][k] with
  // RVV[j] = Phi_diag A+_j Vinv [Nfp][Np] (also the reconstruction of nodal data of side j on
  // the diagonal, Algorithm 2) and GR[j][k] = Dr V A_j A+_k Vinv, GS likewise, [Np][Np].
  std::vector<double> RVV[2], GR[2][2], GS[2][2];
  std::vector<int> hyp;              // [Nfp] rotated-order indices of the shared face's nodes
};

// Builds (and caches) the operators of order N; returns nullptr if N is out of range or the
// reconstruction system is rank deficient (err receives a message).
const RefOps* get_refops(int N, const char** err);

// n-point Gauss-Legendre rule on [-1, 1] (Newton iteration on P_n).
void gauss_legendre_rule(int n, std::vector<double>& x, std::vector<double>& w);

// Orthonormal basis on the reference triangle at (r, s): psi[Np]; optionally gradients.
void simplex_basis(int N, double r, double s, double* psi, double* dpsi_dr, double* dpsi_ds);

}  // namespace rdg
