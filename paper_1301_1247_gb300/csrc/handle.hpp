// Internal state of a built solver (opaque hbs_handle) and of a batch result.
#pragma once

#include <complex>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "devbuf.hpp"

namespace hbs {

// One level of the binary tree (Sec. 4): node-wise index sets I_tau, skeletons,
// interpolation matrices and the Woodbury factors E, F*, G of Eqs. (def_muE..def_muG).
struct Level {
  int l = 0;
  int first = 0;   // heap index of the first node on this level
  int count = 0;   // number of nodes (2^l)
  std::vector<int> n, k;        // |I_tau|, skeleton size |J_tau|
  std::vector<int64_t> off;     // row offset of node tau in the level's index / vector arrays
  int64_t ntot = 0;
  DevBuf<int64_t> idx;          // global boundary indices of I_tau, concatenated
  DevBuf<int> perm;             // pivot order per node (first k = skeleton positions)
  std::vector<int64_t> t_off;   // T = R11^{-1} R12 (k x (n - k)) per node
  DevBuf<cplx> T;
  std::vector<int64_t> e_off, f_off, g_off, dh_off;
  DevBuf<cplx> E, F, G, Dhat;   // E: n x k, F: F* (k x n), G: n x n, Dhat: k x k
  DevBuf<double> cx, cy, rad;   // enclosing circle of the node's original points
  std::vector<double> h_rad;
  // Not compressed (level 1 when the root stays small): P = I, so Dhat = D, E = F* = I and
  // G = 0; the telescoping sweeps pass the level's vectors through unchanged.
  bool passthru = false;
};

// Periodizer blocks on one Sommerfeld contour (Secs. 2.2-2.4).
struct ContourData {
  double t0 = 0.0;
  std::vector<std::complex<double>> k, wk;  // nodes and weights (host)
  DevBuf<cplx> dk, dwk;
  // Columns of W = A^{-1} [B_L | B_R] live in the handle's W buffer at col_off.
  int64_t col_off = 0;
  // Rows: C_L (2M x N) and C_R (2M x N)
  DevBuf<cplx> CL, CR;
  // Wall contributions to the Bragg samples (4 S x 2M for the L and R walls)
  DevBuf<cplx> SL, SR;
  // small products: rows [R_-1; R_1; C_L; C_R; E_-1; E_0; E_1] times columns [W_P | W_BL | W_BR]
  DevBuf<cplx> Zd;  // column-major (zr x zc)
  int zr = 0, zc = 0;
  // Recipes that expand compressed rows (Rsel) / columns (W) to this contour's rows / columns.
  DevBuf<int2> row_recipe, col_recipe;
  // Dense interpolation matrices: C_L = UL C_sel, C_R = UR C_sel (2M x rC);
  // B_L = Y_sel VL^T, B_R = Y_sel VR^T (VL, VR: 2M x rB).
  DevBuf<cplx> UL, UR, VL, VR;
};

struct Handle {
  int64_t N = 0;       // unknowns: boundary nodes x comps
  int64_t nodes = 0;   // boundary nodes
  int comps = 1;       // unknowns per node: 1 (sound-soft) or 2 (transmission, Sec. 5)
  double index = 0.0;  // refractive index n of the obstacles (transmission)
  double d = 1.0, omega = 0.0, tol = 0.0;
  hbs_options opts{};
  int L = 0;
  DevBuf<double> x, y, nx, ny, w;             // per unknown (each node at both of its unknowns)
  std::vector<double> hx, hy, hnx, hny, hw;  // host copies (for host-side planning only)
  std::vector<Level> levels;                  // index = level (0 = root)
  int nroot = 0;
  DevBuf<cplx> Groot;                         // inverse of the root block
  int max_rank = 0;

  // neighbour images (Sec. 3.2): A_{+-1} ~ P_nb R_{+-1}
  int nb_rank = 0;
  double nb_R = 0.0;
  int nb_np = 0;
  DevBuf<int64_t> nb_skel;     // J (l)
  DevBuf<cplx> Pnb;            // N x l
  DevBuf<cplx> Rm, Rp;         // A_{-1}(J,:), A_{+1}(J,:)  (l x N)

  // Bragg sampling
  int S = 0;
  double y0 = 0.0;
  DevBuf<cplx> Esamp;          // 3 images x (4 S x N): rows u(+y0), u(-y0), u_y(+y0), u_y(-y0)

  int M = 0;
  double ch = 0.0, cc = 2.0, cw = 2.0, cK = 0.0;
  std::vector<ContourData> contours;
  int64_t wcols = 0;           // l + rB: columns [P | skeleton columns of B]
  // Interpolative decompositions of the periodizer blocks over all contours:
  //   columns Y = [B_L^0 | B_R^0 | ...] ~ Y(:, JY) [I | TY],  rows C = [C_L^0; C_R^0; ...] and E
  //   ~ rows IC / IE expanded by TC / TE.  Rsel = [R_-1; R_1; C(IC, :); E(IE, :)] (rsel x N).
  int rB = 0, rC = 0, rE = 0, rsel = 0;
  DevBuf<cplx> TY, TC, TE, Rsel;
  DevBuf<cplx> VT;             // (Rsel A^{-1})^T = A^{-T} Rsel^T  (N x rsel)
  DevBuf<cplx> Zc;             // Rsel A^{-1} [P | Y_sel]  (rsel x (l + rB))
  DevBuf<cplx> PE;             // Bragg rows from their skeleton rows (12 S x rE)
  DevBuf<cplx> EZ;             // PE Zc[E rows]  (12 S x (l + rB))
  // V applied to unit plane waves e^{i w (x - c).(cos phi_k, sin phi_k)} at K equispaced
  // directions phi_k = 2 pi k / K (rsel x K); V b(theta) for any incidence angle follows by
  // trigonometric interpolation in theta (the plane wave's Jacobi-Anger expansion is
  // band-limited to |m| <= w max|x - c| + O((w r)^{1/3}) + O(log 1/eps)).
  DevBuf<cplx> Pdir;
  int Kdir = 0;
  double dir_cx = 0.0, dir_cy = 0.0;
  double pid_residual = 0.0;
  double nb_residual = 0.0;     // neighbour ID error on nodes between the candidates

  double build_seconds = 0.0;
  size_t device_bytes() const;
  double factor_bytes = 0.0;
  double apply_flops = 0.0;

  // Guards the dense rows that the plain path forms on first use, so that concurrent
  // solves on one handle stay safe.
  std::mutex lazy_mu;

  void apply_inverse(const cplx* b, cplx* x, int64_t nrhs, cudaStream_t s) const;
  void apply_inverse_transpose(const cplx* b, cplx* x, int64_t nrhs, cudaStream_t s) const;
};

struct AngleResult {
  int n_min = 0, n_max = -1;
  std::vector<std::complex<double>> c, d;
  double flux_err = 0.0;
  int n_wood = 0;
  double t0 = 0.0;
};

struct Result {
  std::vector<AngleResult> angles;
  bool illcond = false;
};

}  // namespace hbs

struct hbs_handle {
  hbs::Handle h;
};
struct hbs_result {
  hbs::Result r;
};
