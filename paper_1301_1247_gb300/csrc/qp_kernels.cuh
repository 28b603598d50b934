// Declarations shared between the library's translation units.
#pragma once

#include <vector>

#include "common.cuh"
#include "handle.hpp"
#include "zgemm.cuh"

namespace hbs {

struct BigQrState {
  int done;
  int rank;
  double r00;
  cplx v0;
  double tau;
};

struct BigQrJobSpec {
  cplx* A;     // m x n, column-major, overwritten
  int64_t m, n;
  int* perm;   // n
  cplx* T;     // output k x (n - k)
};
// Column-pivoted QR / ID of several large matrices at once on all SMs; returns the ranks.
std::vector<int> big_row_id_batched(std::vector<BigQrJobSpec>& specs, double tol, cudaStream_t s);

// pqr.cu: persistent column-pivoted QR (one cooperative launch for all steps of a batch).
struct PqrState {
  int rank;
  int capped;  // stopped at kcap before reaching the tolerance
  double r00;
};
struct PqrSpec {
  cplx* A;       // m x n, column-major (ld m), overwritten by the factorization
  int64_t m, n;
  int kcap;      // largest rank allowed
  int* perm;     // out: n entries, skeleton columns first
  cplx* T;       // out: k x (n - k), ld k (capacity min(m, n, kcap) x n)
};
// Per-step data of the factorizations, concatenated (matrix j at koff[j]): pivot column,
// R diagonal, reflector head and tau; the reflector tail of step s sits in rows s+1..m-1
// of column piv[s] of the factored matrix.
struct PqrOut {
  std::vector<int> rank;
  std::vector<int64_t> koff;
  DevBuf<int> piv;
  DevBuf<cplx> beta, v0;
  DevBuf<double> tau;
};
// equal_steps: the matrices are expected to reach similar ranks (the CTAs are then divided
// by the work of one step); otherwise each is expected to run min(m, n, kcap) steps.
void pqr_run(const std::vector<PqrSpec>& specs, double tol, cudaStream_t s, PqrOut& out, bool equal_steps = false);
// W(:, c) <- R11^{-1} W(:, c) (first k rows) with R11 of matrix `job` of a pqr_run on A (m rows).
void pqr_solve_r11(const cplx* A, int64_t m, const PqrOut& qr, int job, int k, cplx* W, int64_t ldw, int64_t ncols,
                   cudaStream_t s);
// pgj.cu: in-place inverses of several large matrices (pointer, n) in one persistent
// launch; throws HBS_WARN_ILLCOND on a singular block.
void pgj_run(const std::vector<std::pair<cplx*, int>>& mats, cudaStream_t s, const char* what);
// The same by blocked Gauss-Jordan (bgj.cu): panels of columns eliminated by a cluster of
// cs CTAs per block (1, 2, 4 or 8), the rest of each block updated by the batched GEMM.
void bgj_run(const std::vector<std::pair<cplx*, int>>& mats, int cs, cudaStream_t s, const char* what);
// Panel width bgj_run uses for blocks up to nmax on clusters of cs CTAs (0: does not fit).
int bgj_panel_width(int nmax, int cs);
// True for bgj_run's error when the device cannot run the requested cluster shape; the
// blocks are then untouched.
struct Error;
bool bgj_unavailable(const Error& e);
struct InvJob;
// In-place inverses of a batch of blocks (persistent Gauss-Jordan for few or large blocks,
// one CTA per block otherwise); throws HBS_WARN_ILLCOND when a pivot is exactly zero.
void batched_inverse(std::vector<InvJob>& jobs, cudaStream_t s, const char* what);
// X(:, c) = R^{-1} B(:, c) for upper-triangular R (k x k, row-major); X may alias B.
__global__ void k_tsolve_cols(const cplx* R, int k, const cplx* B, int64_t ldb, int64_t ncols, cplx* X, int64_t ldx);
// Columns of conj(Q1), Q1 = the first k columns of the factorization's Q (m x k, ld m).
__global__ void k_form_qc(const cplx* A, int64_t m, const int* piv, const cplx* v0, const double* tau, int k,
                          cplx* Qc);
__global__ void k_r11_rows(const cplx* A, int64_t m, const int* piv, const cplx* beta, int k, cplx* R);
__global__ void k_gather_cols(const cplx* src, int64_t lds, int64_t rows, const int64_t* idx, int64_t ncols, cplx* out,
                              int64_t ldo);
__global__ void k_set_unit_cols(cplx* X, int k, const int64_t* idx);

// persist.cu: the handle to / from a file (HBS_ERR_IO on any file problem)
void save_handle(Handle& h, const char* path, cudaStream_t s);
void load_handle(Handle& h, const char* path, cudaStream_t s);

// hbs_build.cu
void build_hbs(Handle& h, cudaStream_t s);
// Several solvers at once, level by level from the leaves, one launch per kernel and stage.
void build_hbs_multi(const std::vector<Handle*>& hs, cudaStream_t s);
DevGeom Handle_geom(const Handle& h);
void run_gemms(std::vector<GemmJob>& jobs, cudaStream_t s);
// Tensor-core (digit-plane) products of a batch of jobs (ozaki.cu); eligible: large enough
// to pay.
bool ozaki_eligible(const GemmJob& j);
void ozaki_gemm_batched(const std::vector<GemmJob>& jobs, cudaStream_t s);
std::vector<int> batched_id(std::vector<CpqrJob>& jobs, double tol, cudaStream_t s);
__global__ void k_geom(const double* dx, const double* dy, double* nx, double* ny, double* w, int64_t n);

// qp_kernels.cu
__global__ void k_fill_b(DevGeom g, const cplx* k, const cplx* wk, int M, double d, cplx* W, int64_t ldw,
                         int64_t col_bl, int64_t col_br, int combine, cplx alpha);
__global__ void k_fill_c(DevGeom g, const cplx* k, int M, double shift_x, double x0, cplx* C, int64_t ldc);
__global__ void k_fill_samples(DevGeom g, int S, double d, double y0, double shift_x, cplx* E, int64_t lde);
__global__ void k_fill_wall_samples(const cplx* k, const cplx* wk, int M, int S, double d, double y0, double omega,
                                    cplx* SL, cplx* SR);
__global__ void k_fill_nb(DevGeom g, const int64_t* near_m, int nm, const int64_t* near_p, int npn, double d,
                          double cx, double cy, double R, int np, double wp, cplx* Mt);
__global__ void k_fill_r(DevGeom g, const int64_t* J, int l, double d, cplx* Rm, cplx* Rp);
int big_row_id(cplx* Mt, int64_t m, int64_t n, double tol, int* perm, cplx* T, int max_rank, cudaStream_t s);
__global__ void k_bq_norms(const cplx* A, int64_t m, int64_t n, double* nrm, double* nref, int* perm);
__global__ void k_bq_argmax(const double* nrm, int64_t s, int64_t n, const BigQrState* st, double* pv, int* pi);
__global__ void k_bq_pivot(cplx* A, int64_t m, int64_t s, double* nrm, double* nref, int* perm, const double* pv,
                           const int* pi, int nparts, BigQrState* st, double tol);
__global__ void k_bq_update(cplx* A, int64_t m, int64_t n, int64_t s, double* nrm, double* nref,
                            const BigQrState* st);
__global__ void k_bq_tsolve(const cplx* A, int64_t m, int64_t n, int k, cplx* T);

struct ContourPtrs {
  const cplx* k[2];   // contour nodes of contour 0 and (if present) 1
  const cplx* wk[2];  // their weights
  const cplx* s[2];   // sqrt(w - k) sqrt(w + k) at the nodes (principal roots)
  const cplx* si[2];  // 1 / s
};
// s and 1/s at M contour nodes (the wall entries' per-node factors, formed once).
__global__ void k_contour_s(const cplx* k, int M, double omega, cplx* s, cplx* si);
__global__ void k_fill_family_sub(DevGeom g, ContourPtrs cp, int M, double d, int S, double y0, int family,
                                  const int64_t* pts, int np, int nfam, cplx* out, int64_t ld);
__global__ void k_fill_family_sel(DevGeom g, ContourPtrs cp, int M, double d, int S, double y0, int family,
                                  const int* sel, int nsel, cplx* out, int64_t ld);

struct RowRef {
  const cplx* base;  // first element of the row
  int64_t ld;        // stride between consecutive columns
};
__global__ void k_gather_subrows(const cplx* src, int64_t lds, const int64_t* sub, int ns, int ncol, cplx* out,
                                 int64_t ldo);
__global__ void k_gather_subcols_t(const cplx* src, int64_t lds, int nrows, const int64_t* sub, int ns, cplx* out,
                                   int64_t ldo, int col0);
__global__ void k_gather_rowrefs(const RowRef* refs, int nsel, int64_t ncol, cplx* out, int64_t ldo);
__global__ void k_expand_rows(const cplx* in, int64_t ldi, int ncol, const int2* recipe, int nout, const cplx* T1,
                              int r1, int off1, const cplx* T2, int r2, int off2, cplx* out, int64_t ldo);
__global__ void k_expand_cols(const cplx* in, int64_t ldi, int nrow, const int2* recipe, int nout, const cplx* T, int r,
                              int off, const int* skel, cplx* out, int64_t ldo);
__global__ void k_fill_dirs(DevGeom g, double cx, double cy, int K, cplx* out);
__global__ void k_transpose(const cplx* in, int64_t rows, int64_t cols, cplx* out);
__global__ void k_diff_norm2(const cplx* a, int64_t lda, const cplx* b, int64_t ldb, int nrow, int ncol, double* acc);

// qp_solve.cu
// The periodizer and the angle-independent precompute.  With with_hbs, the HBS compression
// and inversion (build_hbs) runs meanwhile on a second stream from a worker thread: the
// neighbour and periodizer IDs and the selected rows depend on the geometry only, and the
// two share the device until the transposed sweep, which needs both.
void build_periodizer(Handle& h, cudaStream_t s, bool with_hbs = false);
void solve_angles(Handle& h, const double* theta, int64_t n_theta, bool plain, Result& out, cudaStream_t s);
// The same angles with the proxy-point / wall-discrepancy periodizer (proxy.cu).
void solve_angles_proxy(Handle& h, const double* theta, int64_t n_theta, Result& out, cudaStream_t s);

inline int grid_1d(int64_t tot, int nt = 256, int cap = 8192) {
  int64_t b = (tot + nt - 1) / nt;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

}  // namespace hbs
