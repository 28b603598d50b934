// Periodizer precompute and the per-Bloch-phase block solve (Secs. 2.2-2.4, 3).
//
// With the neighbour factors A_{+-1} ~ P R_{+-1} (Sec. 3.2), Eq. (block2) becomes the
// extended system
//     [ A   L   B   PW ] [eta ]   [b]        L = [alpha^{-1} P | alpha P],  R = [R_{-1}; R_1]
//     [ R  -I   0   0  ] [zeta] = [0]        B = B_L + alpha B_R
//     [ C~  0   Q   0  ] [xi  ]   [0]        C~ = alpha C_L - alpha^{-2} C_R  (P = 1)
//     [ Wr  0   Wx  Wa ] [a   ]   [0]        Wood's rows/columns (Sec. 2.4)
// Eliminating eta = A^{-1}(b - L zeta - B xi - PW a) leaves a Schur system in
// (zeta, xi, a) of size 2l + 2M + n_wood (Eqs. blocksolve and inv).  Every product it
// needs is "a row functional of A^{-1} times a column": rows R, C_L, C_R and the Bragg
// sampling rows E; columns P, B_L, B_R (angle independent, applied once at build:
// W = A^{-1}[P | B_L | B_R], Z = Rows W) and the right-hand sides b, PW (per Bloch phase:
// X = A^{-1}[b | PW], Proj = Rows X).  The plain path applies A^{-1} to L and B(alpha)
// for every Bloch phase instead, q + 2M + 2l applies (Remark 3.2).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <exception>
#include <map>
#include <mutex>
#include <thread>
#include <type_traits>

#include "dense_kernels.cuh"
#include "dfloat.cuh"
#include "profile.hpp"
#include "gridsync.cuh"
#include "qp_kernels.cuh"
#include "tune.hpp"

namespace hbs {

using zc = std::complex<double>;

__global__ void k_dense_from_recipe(const int2* rec, int nout, int tkind, const cplx* T, int r, int off, cplx* out);

static inline cplx to_c(zc v) { return cmk(v.real(), v.imag()); }

// ---------------------------------------------------------------------------
// Periodizer precompute
// ---------------------------------------------------------------------------

static void contour_nodes(ContourData& c, int M, double h, double cc, double cw, double t0) {
  c.t0 = t0;
  c.k.resize(M);
  c.wk.resize(M);
  for (int m = 0; m < M; ++m) {
    double t = t0 + (m - 0.5 * (M - 1)) * h;
    double u = (t - t0) / cw;
    double ch = std::cosh(u);
    c.k[m] = zc(t, -cc * std::tanh(u));
    c.wk[m] = zc(h, -h * (cc / cw) / (ch * ch));
  }
  std::vector<cplx> kk(M), ww(M);
  for (int m = 0; m < M; ++m) { kk[m] = to_c(c.k[m]); ww[m] = to_c(c.wk[m]); }
  c.dk.upload(kk, 0);
  c.dwk.upload(ww, 0);
}

// Pole-free crossing point for angles at or near a Wood's anomaly: half the smallest
// positive k_n that occurs at an exact anomaly, k = sqrt(w^2 - (w - 2 pi j / d)^2).
static double auto_wood_shift(double omega, double d) {
  double best = 1e300;
  for (int j = 1; 2.0 * M_PI * j / d < 2.0 * omega; ++j) {
    double kap = omega - 2.0 * M_PI * j / d;
    double v = omega * omega - kap * kap;
    if (v > 1e-12) best = std::min(best, std::sqrt(v));
  }
  if (best > 1e299) best = omega;
  return 0.5 * best;
}

// Distance, in the contour variable t, from a pole p of the wall integrands to the
// Sommerfeld contour k(t) = t - i c tanh((t - t0)/w): min |k(t) - p| / |k'(t)| over a fine
// sampling of t around the contour's bend (far from it the contour runs at |Im k| = c and
// only nearby poles can come close).
static double contour_distance(const Handle& h, int c, std::complex<double> p) {
  const double t0 = h.contours[c].t0, cc = h.cc, cw = h.cw;
  if (std::fabs(p.imag()) > cc + 3.0) return 1e300;
  double best = 1e300;
  // k(t) = t + O(c), so the nearest contour point lies within a few units of Re p in t
  const double lo = p.real() - 4.0, hi = p.real() + 4.0;
  for (double t = lo; t <= hi; t += 0.02) {
    const double u = (t - t0) / cw;
    const double th = std::tanh(u), sech2 = 1.0 - th * th;
    const std::complex<double> k(t, -cc * th);
    const double dk = std::hypot(1.0, cc / cw * sech2);
    best = std::min(best, std::abs(k - p) / dk);
  }
  return best;
}

namespace {
// Runs build_hbs on its own stream from a worker thread (same device and arithmetic modes
// as the caller); join() waits for it and rethrows its error.  The destructor joins too,
// so an error on the calling thread never leaves the worker running.
struct HbsWorker {
  std::thread t;
  cudaStream_t s2 = nullptr;
  std::exception_ptr err;
  void start(Handle& h) {
    int dev = 0;
    HBS_CUDA(cudaGetDevice(&dev));
    // The compression and inversion are the longer of the two concurrent chains: their
    // CTAs are scheduled ahead of the periodizer's whenever both are waiting.
    int least = 0, greatest = 0;
    HBS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    HBS_CUDA(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, greatest));
    const bool df = gemm_double_float(), tc = gemm_tensor();
    t = std::thread([this, &h, dev, df, tc] {
      try {
        HBS_CUDA(cudaSetDevice(dev));
        gemm_double_float() = df;
        gemm_tensor() = tc;
        StreamScope scope(s2);
        {
          prof::Phase ph("build:hbs_compress_invert", s2);
          build_hbs(h, s2);
        }
        HBS_CUDA(cudaStreamSynchronize(s2));
      } catch (...) {
        err = std::current_exception();
      }
    });
  }
  void join() {
    if (t.joinable()) t.join();
    if (s2) {
      cudaStreamDestroy(s2);
      s2 = nullptr;
    }
    if (err) {
      std::exception_ptr e = err;
      err = nullptr;
      std::rethrow_exception(e);
    }
  }
  ~HbsWorker() {
    if (t.joinable()) t.join();
    if (s2) cudaStreamDestroy(s2);
  }
};
}  // namespace

namespace {
// Marks this thread as the background chain while the compression runs beside it.
struct BackgroundScope {
  bool prev;
  explicit BackgroundScope(bool on) : prev(background_chain()) { background_chain() = on || prev; }
  void end() { background_chain() = prev; }
  ~BackgroundScope() { end(); }
};
}  // namespace

void build_periodizer(Handle& h, cudaStream_t s, bool with_hbs) {
  HbsWorker hbs_worker;
  if (with_hbs) hbs_worker.start(h);
  BackgroundScope background(with_hbs);
  const int64_t N = h.N;
  const DevGeom g = Handle_geom(h);
  const double d = h.d, omega = h.omega;

  // ---- geometry extents (host planning)
  double cx = 0, cy = 0;
  {
    double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300;
    for (int64_t i = 0; i < N; ++i) {
      mnx = std::min(mnx, h.hx[i]); mxx = std::max(mxx, h.hx[i]);
      mny = std::min(mny, h.hy[i]); mxy = std::max(mxy, h.hy[i]);
    }
    cx = 0.5 * (mnx + mxx);
    cy = 0.5 * (mny + mxy);
  }
  double rmax = 0.0, ymax = 0.0, xmax = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    rmax = std::max(rmax, std::hypot(h.hx[i] - cx, h.hy[i] - cy));
    ymax = std::max(ymax, std::fabs(h.hy[i]));
    xmax = std::max(xmax, std::fabs(h.hx[i]));
  }
  double rsrc = 1e300;
  for (int64_t i = 0; i < N; ++i) {
    rsrc = std::min(rsrc, std::hypot(h.hx[i] - d - cx, h.hy[i] - cy));
    rsrc = std::min(rsrc, std::hypot(h.hx[i] + d - cx, h.hy[i] - cy));
  }

  prof::PhaseSeq ph(s);
  ph.next("build:periodizer_fill");

  // ---- Sommerfeld contours (Sec. 2.3)
  h.cc = h.opts.contour_c > 0 ? h.opts.contour_c : 2.0;
  h.cw = h.opts.contour_w > 0 ? h.opts.contour_w : 2.0;
  // Trapezoid spacing: a pole of the wall integrands at distance delta (in t) from the
  // contour costs about exp(-2 pi delta / h); over all incidence angles the nearer of the
  // two contours keeps delta >= ~0.75, so h = 0.2 holds the quadrature error near 1e-10.
  h.ch = h.opts.contour_h > 0 ? h.opts.contour_h : 0.2;
  double shift = h.opts.wood_shift;
  if (shift == 0.0) shift = auto_wood_shift(omega, d);
  {
    const double dB = 0.5 * d - xmax, dC = 1.5 * d - xmax;
    const double smin = 37.0 / (dB + dC);
    double K = h.opts.contour_k > 0 ? h.opts.contour_k : std::sqrt(omega * omega + smin * smin) + 2.0 * h.cw;
    if (shift > 0) K += shift;
    h.cK = K;
  }
  h.M = h.opts.m > 0 ? h.opts.m : (int)std::ceil(2.0 * h.cK / h.ch);
  const int M = h.M;
  const int nc = shift > 0 ? 2 : 1;
  h.contours.clear();
  h.contours.resize(nc);
  for (int c = 0; c < nc; ++c) contour_nodes(h.contours[c], M, h.ch, h.cc, h.cw, c == 0 ? 0.0 : shift);

  // ---- Bragg sampling rows (Remarks 2.2, 2.3)
  h.S = h.opts.n_bragg_samples > 0 ? h.opts.n_bragg_samples
                                   : std::max(32, 2 * (int)std::ceil(omega * d / (2.0 * M_PI)) + 44);
  h.y0 = h.opts.y0 > 0 ? h.opts.y0 : ymax + 0.25 * d;
  const int S = h.S;
  // (the full sampling rows E and wall rows C are only formed for the plain path, on demand)

  // ---- contours' wall-sample rows (small: 4S x 2M each)
  const int ny = 4 * M * nc;
  ContourPtrs cp{};
  DevBuf<cplx> cs_tab[2], csi_tab[2];
  for (int c = 0; c < nc; ++c) {
    ContourData& cd = h.contours[c];
    cd.col_off = (int64_t)4 * M * c;
    cp.k[c] = cd.dk.get();
    cp.wk[c] = cd.dwk.get();
    cs_tab[c].alloc(M);
    csi_tab[c].alloc(M);
    k_contour_s<<<(M + 255) / 256, 256, 0, s>>>(cd.dk.get(), M, omega, cs_tab[c].get(), csi_tab[c].get());
    cp.s[c] = cs_tab[c].get();
    cp.si[c] = csi_tab[c].get();
    cd.SL.alloc((size_t)4 * S * 2 * M);
    cd.SR.alloc((size_t)4 * S * 2 * M);
    {
      prof::KScope _ks("k_fill_wall_samples", s);
      k_fill_wall_samples<<<grid_1d((int64_t)4 * S * M), 256, 0, s>>>(cd.dk.get(), cd.dwk.get(), M, S, d, h.y0, omega,
                                                                       cd.SL.get(), cd.SR.get());
    }
    HBS_LAUNCH_CHECK("k_fill_wall_samples");
  }

  // ---- interpolative decompositions of the periodizer blocks on a subsample of points:
  // family 0 = columns of Y = [B_L^c | B_R^c ...], 1 = rows of C = [C_L^c; C_R^c ...],
  // 2 = the Bragg sampling rows E.  Their members are smooth functions of the boundary
  // node, so an ID found on a fine subsample holds on all N nodes; a disjoint second
  // subsample checks that.
  ph.next("build:periodizer_id");
  // Subsample size: at least 12 points per oscillation of the fastest member along the
  // boundary (wavenumbers up to the contour's reach cK), never fewer than 512 (at w = 60,
  // ~40 oscillations: 512 nodes against family ranks of at most ~200); a family's sampled
  // matrix then stays resident in L2 through the ID's steps.
  double perim = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const int64_t j = (i + 1) % N;
    perim += std::hypot(h.hx[j] - h.hx[i], h.hy[j] - h.hy[i]);
  }
  const double osc = perim * std::max(omega, h.cK) / (2.0 * M_PI);
  int ns_want = std::max(512, (int)std::ceil(12.0 * osc / 256.0) * 256);
  // subsamples of whole nodes (both unknowns of a transmission node)
  const int comps = h.comps;
  const int64_t nodes = N / comps;
  const int nsn = (int)std::min<int64_t>(nodes, std::min(ns_want, 16384));
  // check sample: half as many nodes, each half-way between two nodes of the subsample
  const int ns2n = std::max(1, nsn / 2);
  const int ns = nsn * comps, ns2 = ns2n * comps;
  std::vector<int64_t> hsub(ns), hsub2(ns2);
  for (int i = 0; i < nsn; ++i)
    for (int u = 0; u < comps; ++u) hsub[i * comps + u] = (int64_t)((double)i * nodes / nsn) * comps + u;
  for (int i = 0; i < ns2n; ++i)
    for (int u = 0; u < comps; ++u)
      hsub2[i * comps + u] =
          std::min<int64_t>(nodes - 1, (int64_t)(((double)(2 * i) + 0.5) * nodes / nsn)) * comps + u;
  DevBuf<int64_t> dsub, dsub2;
  dsub.upload(hsub, s);
  dsub2.upload(hsub2, s);
  const double ptol = std::min(0.1 * h.tol, 1e-13);
  const int nce = 12 * S;
  // IDs: returns rank, fills perm (host), T (device), and the check residual on the second subsample.
  // The three families' IDs run in one persistent QR launch (one after another they took
  // longer: their pivot steps then add up); each is then checked on the second subsample
  // (members rebuilt from the skeleton members).
  struct Family {
    int family, ncols;
    DevBuf<cplx> A, A2, T;
    DevBuf<int> perm;
  };
  Family fams[3];
  fams[0].family = 0; fams[0].ncols = ny;
  fams[1].family = 1; fams[1].ncols = ny;
  fams[2].family = 2; fams[2].ncols = nce;
  std::vector<PqrSpec> fspecs;
  for (Family& f : fams) {
    const int ncols = f.ncols;
    f.A.alloc((size_t)ns * ncols);
    f.A2.alloc((size_t)ns2 * ncols);
    {
      prof::KScope _ks("k_fill_family_sub", s);
      k_fill_family_sub<<<grid_1d((int64_t)ns * ncols), 256, 0, s>>>(g, cp, M, d, S, h.y0, f.family, dsub.get(), ns,
                                                                      ncols, f.A.get(), ns);
      k_fill_family_sub<<<grid_1d((int64_t)ns2 * ncols), 256, 0, s>>>(g, cp, M, d, S, h.y0, f.family, dsub2.get(),
                                                                       ns2, ncols, f.A2.get(), ns2);
    }
    HBS_LAUNCH_CHECK("k_fill_family_sub");
    f.perm.alloc(ncols);
    f.T.alloc((size_t)std::min(ns, ncols) * ncols);
    fspecs.push_back({f.A.get(), ns, ncols, std::min(ns, ncols), f.perm.get(), f.T.get()});
  }
  PqrOut fqr;
  pqr_run(fspecs, ptol, s, fqr, /*equal_steps=*/true);  // family ranks are alike (~100-200 at w = 60)
  int fqr_rank[3];
  for (int fi = 0; fi < 3; ++fi) fqr_rank[fi] = fqr.rank[fi];
  h.pid_residual = 0.0;
  std::vector<int> fperm[3];
  DevBuf<cplx>* Touts[3] = {&h.TY, &h.TC, &h.TE};
  int franks[3];
  for (int fi = 0; fi < 3; ++fi) {
    Family& f = fams[fi];
    const int ncols = f.ncols, r = fqr_rank[fi];
    franks[fi] = r;
    std::vector<int>& hperm = fperm[fi];
    hperm = f.perm.download(s);
    DevBuf<cplx>& Tout = *Touts[fi];
    Tout.alloc(std::max<int64_t>((int64_t)r * (ncols - r), 1));
    if ((int64_t)r * (ncols - r) > 0)
      HBS_CUDA(cudaMemcpyAsync(Tout.get(), f.T.get(), sizeof(cplx) * r * (ncols - r), cudaMemcpyDeviceToDevice, s));
    std::vector<int2> rec(ncols);
    std::vector<int> inv(ncols);
    for (int p = 0; p < ncols; ++p) inv[hperm[p]] = p;
    for (int a = 0; a < ncols; ++a) rec[a] = inv[a] < r ? make_int2(0, a) : make_int2(1, inv[a] - r);
    DevBuf<int2> drec;
    drec.upload(rec, s);
    DevBuf<int> dperm;
    dperm.upload(hperm, s);
    DevBuf<cplx> B2((size_t)ns2 * ncols);
    {
      prof::KScope _ks("k_expand_cols", s);
      k_expand_cols<<<grid_1d((int64_t)ns2 * ncols), 256, 0, s>>>(f.A2.get(), ns2, ns2, drec.get(), ncols, Tout.get(),
                                                                   r, 0, dperm.get(), B2.get(), ns2);
    }
    DevBuf<double> acc(2);
    HBS_CUDA(cudaMemsetAsync(acc.get(), 0, 2 * sizeof(double), s));
    {
      prof::KScope _ks("k_diff_norm2", s);
      k_diff_norm2<<<grid_1d((int64_t)ns2 * ncols), 256, 0, s>>>(B2.get(), ns2, f.A2.get(), ns2, ns2, ncols, acc.get());
    }
    auto ha = acc.download(s);
    const double res = ha[1] > 0 ? std::sqrt(ha[0] / ha[1]) : 0.0;
    h.pid_residual = std::max(h.pid_residual, res);
  }
  std::vector<int>& permY = fperm[0];
  std::vector<int>& permC = fperm[1];
  std::vector<int>& permE = fperm[2];
  h.rB = franks[0];
  h.rC = franks[1];
  h.rE = franks[2];
  HBS_LAUNCH_CHECK("periodizer ids");

  // ---- neighbour interactions (after the periodizer: with the compression running beside
  // this thread, the periodizer's large persistent QR then overlaps the leaf levels, whose
  // kernels are not cooperative, instead of a level that waits for the cooperative-launch lock)
  ph.next("build:neighbour_id");
  // ---- neighbour proxy circle and near points (Sec. 3.2)
  double R = h.opts.nb_radius;
  if (!(R > 0.0)) R = rsrc > 1.05 * rmax ? 0.5 * (rmax + rsrc) : 1.1 * rmax;
  std::vector<int64_t> near_m, near_p;
  double rfar = 1e300;
  for (int64_t i = 0; i < N; ++i) {
    double dm = std::hypot(h.hx[i] - d - cx, h.hy[i] - cy);
    double dp = std::hypot(h.hx[i] + d - cx, h.hy[i] - cy);
    if (dm < R) near_m.push_back(i); else rfar = std::min(rfar, dm);
    if (dp < R) near_p.push_back(i); else rfar = std::min(rfar, dp);
  }
  int np = h.opts.nb_proxies;
  if (np <= 0) {
    // The fields of image sources beyond r_far restricted to the obstacle (radius r_max)
    // have Fourier-Bessel modes decaying like (r_max / r_far)^|m| past |m| ~ w R; the
    // proxy circle must span modes up to that cut-off (an ID needs the span only).
    double q = std::min(rmax / rfar, 0.97);
    np = (int)(2.0 * (std::ceil(omega * R) + std::ceil(std::log(1e-16) / std::log(q)) + 8));
    np = std::max(64, std::min(np, 2048));
    np = (np + 7) / 8 * 8;
  }
  const double wp = 2.0 * M_PI * R / np;
  h.nb_R = R;
  h.nb_np = np;
  {
    const int nm = (int)near_m.size(), npn = (int)near_p.size();
    const int64_t m = nm + npn + np;
    DevBuf<int64_t> dnm, dnp;
    dnm.upload(near_m, s);
    dnp.upload(near_p, s);
    DevBuf<cplx> Mt(m * N);
    {
      prof::KScope _ks("k_fill_nb", s);
      const size_t dsm = 2 * (size_t)np * sizeof(double);
      HBS_CUDA(raise_smem_limit((const void*)k_fill_nb, dsm));
      k_fill_nb<<<grid_1d(m * N), 256, dsm, s>>>(g, dnm.get(), nm, dnp.get(), npn, d, cx, cy, R, np, wp, Mt.get());
    }
    HBS_LAUNCH_CHECK("k_fill_nb");
    // Row ID of the neighbour interactions (Def. 3.1).  The skeleton is chosen by a
    // column-pivoted QR among at most 4096 candidate boundary nodes (every stride-th): their
    // columns of Mt are smooth functions of the node, so candidates far finer than the
    // wavelength lose nothing.  Every node's interpolation coefficients then follow by
    // least squares against the skeleton columns, t_i = R11^{-1} Q1^H Mt(:, i), which for
    // the candidates is exactly T = R11^{-1} R12 of the QR.
    // Candidates are whole nodes (both unknowns of a transmission node, whose rows differ).
    const int comps = h.comps;
    const int64_t nodes = N / comps;
    const int64_t stride = std::max<int64_t>(1, (N + 4095) / 4096);
    const int64_t ncn = (nodes + stride - 1) / stride;  // candidate nodes
    const int64_t nc = ncn * comps;
    DevBuf<cplx> Mc((size_t)m * nc);
    std::vector<int64_t> cand(nc);
    for (int64_t c = 0; c < ncn; ++c)
      for (int u = 0; u < comps; ++u) cand[c * comps + u] = c * stride * comps + u;
    if (comps == 1) {
      HBS_CUDA(cudaMemcpy2DAsync(Mc.get(), sizeof(cplx) * m, Mt.get(), sizeof(cplx) * m * stride, sizeof(cplx) * m,
                                 nc, cudaMemcpyDeviceToDevice, s));
    } else {
      DevBuf<int64_t> dcand;
      dcand.upload(cand, s);
      prof::KScope _ks("k_gather_cols", s);
      k_gather_cols<<<grid_1d(m * nc), 256, 0, s>>>(Mt.get(), m, m, dcand.get(), nc, Mc.get(), m);
      HBS_CUDA(cudaStreamSynchronize(s));  // dcand goes out of scope
    }
    const int kcap = (int)std::min<int64_t>(std::min<int64_t>(m, nc), 4096);
    DevBuf<int> cperm(nc);
    PqrOut qr;
    {
      std::vector<PqrSpec> sp{{Mc.get(), m, nc, kcap, cperm.get(), nullptr}};
      pqr_run(sp, h.tol, s, qr);
    }
    const int l = qr.rank[0];
    h.nb_rank = l;
    std::vector<int> hpiv = qr.piv.download(s, l);
    std::vector<int64_t> J(l);
    for (int i = 0; i < l; ++i) J[i] = cand[hpiv[i]];
    h.nb_skel.upload(J, s);
    h.Rm.alloc(std::max<int64_t>((int64_t)l * N, 1));
    h.Rp.alloc(std::max<int64_t>((int64_t)l * N, 1));
    h.Pnb.alloc(std::max<int64_t>((int64_t)l * N, 1));
    h.nb_residual = 0.0;
    if (l > 0) {
      {
        prof::KScope _ks("k_fill_r", s);
        k_fill_r<<<grid_1d((int64_t)l * N), 256, 0, s>>>(g, h.nb_skel.get(), l, d, h.Rm.get(), h.Rp.get());
      }
      HBS_LAUNCH_CHECK("k_fill_r");
      DevBuf<cplx> Qc((size_t)m * l), Tall((size_t)l * N);
      {
        prof::KScope _ks("k_form_qc", s);
        k_form_qc<<<l, 256, 0, s>>>(Mc.get(), m, qr.piv.get(), qr.v0.get(), qr.tau.get(), l, Qc.get());
      }
      HBS_LAUNCH_CHECK("neighbour Q1");
      // Tall = Q1^H Mt (l x N), then R11^{-1} in place; skeleton nodes get unit columns.
      std::vector<GemmJob> gj(1);
      gj[0] = GemmJob{Qc.get(), Mt.get(), Tall.get(), l, (int)N, (int)m, (int)m, (int)m, l,
                      cmk(1.0, 0.0), cmk(0.0, 0.0), 0, 0, 0, 1};
      run_gemms(gj, s);
      pqr_solve_r11(Mc.get(), m, qr, 0, l, Tall.get(), l, N, s);
      {
        prof::KScope _ks("k_set_unit_cols", s);
        k_set_unit_cols<<<grid_1d((int64_t)l * l), 256, 0, s>>>(Tall.get(), l, h.nb_skel.get());
      }
      {
        prof::KScope _ks("k_transpose", s);
        k_transpose<<<grid_1d((int64_t)l * N), 256, 0, s>>>(Tall.get(), l, N, h.Pnb.get());
      }
      HBS_LAUNCH_CHECK("neighbour interpolation");
      // Check on nodes half-way between candidates: |Mt(:, i) - Mt(:, J) t_i| / |Mt(:, i)|.
      if (stride > 1) {
        const int64_t nchk_n = std::min<int64_t>(ncn - 1, 4096 / comps);
        const int64_t nchk = nchk_n * comps;
        std::vector<int64_t> chk(nchk);
        for (int64_t c = 0; c < nchk_n; ++c) {
          const int64_t node = std::min<int64_t>(nodes - 1, ((c * (ncn - 1)) / nchk_n) * stride + stride / 2);
          for (int u = 0; u < comps; ++u) chk[c * comps + u] = node * comps + u;
        }
        DevBuf<int64_t> dchk;
        dchk.upload(chk, s);
        DevBuf<cplx> G((size_t)m * l), Ms((size_t)m * nchk), Ts((size_t)l * nchk), Rec((size_t)m * nchk);
        {
          prof::KScope _ks("k_gather_cols", s);
          k_gather_cols<<<grid_1d((int64_t)m * l), 256, 0, s>>>(Mt.get(), m, m, h.nb_skel.get(), l, G.get(), m);
          k_gather_cols<<<grid_1d(m * nchk), 256, 0, s>>>(Mt.get(), m, m, dchk.get(), nchk, Ms.get(), m);
          k_gather_cols<<<grid_1d((int64_t)l * nchk), 256, 0, s>>>(Tall.get(), l, l, dchk.get(), nchk, Ts.get(), l);
        }
        std::vector<GemmJob> cj(1);
        cj[0] = GemmJob{G.get(), Ts.get(), Rec.get(), (int)m, (int)nchk, l, (int)m, l, (int)m,
                        cmk(1.0, 0.0), cmk(0.0, 0.0), 0, 0, 0, 0};
        run_gemms(cj, s);
        DevBuf<double> acc(2);
        HBS_CUDA(cudaMemsetAsync(acc.get(), 0, 2 * sizeof(double), s));
        {
          prof::KScope _ks("k_diff_norm2", s);
          k_diff_norm2<<<grid_1d(m * nchk), 256, 0, s>>>(Rec.get(), m, Ms.get(), m, (int)m, (int)nchk, acc.get());
        }
        auto ha = acc.download(s);
        h.nb_residual = ha[1] > 0 ? std::sqrt(ha[0] / ha[1]) : 0.0;
      }
    }
    HBS_CUDA(cudaStreamSynchronize(s));
  }
  const int l = h.nb_rank;

  // ---- source columns [P | Y(:, JY)] (not applied: Z is formed as V [P | Y_sel])
  ph.next("build:skeleton_columns");
  const int rB = h.rB, rC = h.rC, rE = h.rE;
  h.wcols = l + rB;
  DevBuf<cplx> Csrc((size_t)N * h.wcols);
  {
    if (l > 0) HBS_CUDA(cudaMemcpyAsync(Csrc.get(), h.Pnb.get(), sizeof(cplx) * N * l, cudaMemcpyDeviceToDevice, s));
    if (rB > 0) {
      DevBuf<int> jy;
      jy.upload(std::vector<int>(permY.begin(), permY.begin() + rB), s);
      prof::KScope _ks("k_fill_family_sel", s);
      k_fill_family_sel<<<grid_1d(N * (int64_t)rB), 256, 0, s>>>(g, cp, M, d, S, h.y0, 0, jy.get(), rB,
                                                                  Csrc.get() + (int64_t)l * N, N);
      HBS_CUDA(cudaStreamSynchronize(s));
    }
  }

  // ---- Rsel = [R_-1; R_1; C(IC, :); E(IE, :)] and Z = Rsel W
  ph.next("build:R_rows");
  h.rsel = 2 * l + rC + rE;
  {
    h.Rsel.alloc((size_t)h.rsel * N);
    std::vector<RowRef> refs;
    for (int i = 0; i < l; ++i) refs.push_back({h.Rm.get() + i, l});
    for (int i = 0; i < l; ++i) refs.push_back({h.Rp.get() + i, l});
    DevBuf<RowRef> drefs;
    drefs.upload(refs, s);
    if (l > 0) {
      prof::KScope _ks("k_gather_rowrefs", s);
      k_gather_rowrefs<<<grid_1d((int64_t)2 * l * N), 256, 0, s>>>(drefs.get(), 2 * l, N, h.Rsel.get(), h.rsel);
    }
    DevBuf<int> ic, ie;
    ic.upload(std::vector<int>(permC.begin(), permC.begin() + rC), s);
    ie.upload(std::vector<int>(permE.begin(), permE.begin() + rE), s);
    {
      prof::KScope _ks("k_fill_family_sel", s);
      if (rC > 0)
        k_fill_family_sel<<<grid_1d(N * (int64_t)rC), 256, 0, s>>>(g, cp, M, d, S, h.y0, 1, ic.get(), rC,
                                                                    h.Rsel.get() + 2 * l, h.rsel);
      if (rE > 0)
        k_fill_family_sel<<<grid_1d(N * (int64_t)rE), 256, 0, s>>>(g, cp, M, d, S, h.y0, 2, ie.get(), rE,
                                                                    h.Rsel.get() + 2 * l + rC, h.rsel);
    }
    HBS_LAUNCH_CHECK("Rsel fills");
    HBS_CUDA(cudaStreamSynchronize(s));
  }
  // ---- V^T = A^{-T} Rsel^T (one transposed apply of the compressed inverse)
  if (with_hbs) {
    ph.next("build:wait_hbs");
    hbs_worker.join();  // the compressed inverse is complete
    background.end();
  }
  ph.next("build:V_apply");
  h.VT.alloc((size_t)N * h.rsel);
  {
    DevBuf<cplx> RT((size_t)N * h.rsel);
    {
      prof::KScope _ks("k_transpose", s);
      k_transpose<<<grid_1d((int64_t)N * h.rsel), 256, 0, s>>>(h.Rsel.get(), h.rsel, N, RT.get());
    }
    HBS_LAUNCH_CHECK("k_transpose");
    // all rows in one sweep (the level vectors take about 3 N rsel complex values): one
    // batch of products per level instead of one per chunk
    const int64_t chunk = 1024;
    for (int64_t c0 = 0; c0 < h.rsel; c0 += chunk) {
      int64_t nq = std::min<int64_t>(chunk, h.rsel - c0);
      h.apply_inverse_transpose(RT.get() + c0 * N, h.VT.get() + c0 * N, nq, s);
    }
  }
  ph.next("build:Z_products");
  DevBuf<cplx> Zc((size_t)h.rsel * h.wcols);
  {
    std::vector<GemmJob> gj(1);
    gj[0] = {h.VT.get(), Csrc.get(), Zc.get(), h.rsel, (int)h.wcols, (int)N, (int)N, (int)N, h.rsel, cmk(1, 0),
             cmk(0, 0), 0, 0, 0, 1};
    run_gemms(gj, s);
  }
  Csrc.release();
  // interpolation matrices of the reduced Schur systems
  std::vector<int> invC(ny), invE(nce), invY(ny);
  for (int p = 0; p < ny; ++p) invC[permC[p]] = p;
  for (int p = 0; p < nce; ++p) invE[permE[p]] = p;
  for (int p = 0; p < ny; ++p) invY[permY[p]] = p;
  const int zr = 2 * l + 4 * M + 12 * S, zcn = l + 4 * M;
  for (int c = 0; c < nc; ++c) {
    ContourData& cd = h.contours[c];
    cd.zr = zr;
    cd.zc = zcn;
    std::vector<int2> rrec(zr), crec(zcn);
    for (int o = 0; o < 2 * l; ++o) rrec[o] = make_int2(0, o);
    for (int j = 0; j < 4 * M; ++j) {
      const int p = invC[4 * M * c + j];
      rrec[2 * l + j] = p < rC ? make_int2(0, 2 * l + p) : make_int2(1, p - rC);
    }
    for (int e = 0; e < nce; ++e) {
      const int p = invE[e];
      rrec[2 * l + 4 * M + e] = p < rE ? make_int2(0, 2 * l + rC + p) : make_int2(2, p - rE);
    }
    for (int j = 0; j < l; ++j) crec[j] = make_int2(0, j);
    for (int j = 0; j < 4 * M; ++j) {
      const int p = invY[4 * M * c + j];
      crec[l + j] = p < rB ? make_int2(0, l + p) : make_int2(1, p - rB);
    }
    cd.row_recipe.upload(rrec, s);
    cd.col_recipe.upload(crec, s);
    cd.UL.alloc((size_t)2 * M * std::max(rC, 1));
    cd.UR.alloc((size_t)2 * M * std::max(rC, 1));
    cd.VL.alloc((size_t)2 * M * std::max(rB, 1));
    cd.VR.alloc((size_t)2 * M * std::max(rB, 1));
    {
      prof::KScope _ks("k_dense_from_recipe", s);
      k_dense_from_recipe<<<grid_1d((int64_t)2 * M * rC), 256, 0, s>>>(cd.row_recipe.get() + 2 * l, 2 * M, 1,
                                                                        h.TC.get(), rC, 2 * l, cd.UL.get());
      k_dense_from_recipe<<<grid_1d((int64_t)2 * M * rC), 256, 0, s>>>(cd.row_recipe.get() + 2 * l + 2 * M, 2 * M, 1,
                                                                        h.TC.get(), rC, 2 * l, cd.UR.get());
      k_dense_from_recipe<<<grid_1d((int64_t)2 * M * rB), 256, 0, s>>>(cd.col_recipe.get() + l, 2 * M, 1, h.TY.get(),
                                                                        rB, l, cd.VL.get());
      k_dense_from_recipe<<<grid_1d((int64_t)2 * M * rB), 256, 0, s>>>(cd.col_recipe.get() + l + 2 * M, 2 * M, 1,
                                                                        h.TY.get(), rB, l, cd.VR.get());
    }
    HBS_LAUNCH_CHECK("interpolation matrices");
    if (c == 0) {
      h.PE.alloc((size_t)nce * std::max(rE, 1));
      {
        prof::KScope _ks("k_dense_from_recipe", s);
        k_dense_from_recipe<<<grid_1d((int64_t)nce * rE), 256, 0, s>>>(cd.row_recipe.get() + 2 * l + 4 * M, nce, 2,
                                                                        h.TE.get(), rE, 2 * l + rC, h.PE.get());
      }
      h.EZ.alloc((size_t)nce * h.wcols);
      std::vector<GemmJob> gj(1);
      gj[0] = {h.PE.get(), Zc.get() + 2 * l + rC, h.EZ.get(), nce, (int)h.wcols, rE, nce, h.rsel, nce, cmk(1, 0),
               cmk(0, 0), 0, 0, 0};
      run_gemms(gj, s);
    }
    HBS_CUDA(cudaStreamSynchronize(s));
  }
  h.Zc = std::move(Zc);

  // ---- V on plane waves in K equispaced incidence directions (interpolated per angle)
  ph.next("build:direction_samples");
  {
    double rdir = 0.0;
    for (int64_t i = 0; i < N; ++i) rdir = std::max(rdir, std::hypot(h.hx[i] - cx, h.hy[i] - cy));
    const double wr = omega * rdir;
    int K = 2 * (int)std::ceil(wr + 10.0 * std::cbrt(wr) + 30.0);
    K = (K + 31) / 32 * 32;
    h.Kdir = K;
    h.dir_cx = cx;
    h.dir_cy = cy;
    DevBuf<cplx> src((size_t)N * K);
    {
      prof::KScope _ks("k_fill_dirs", s);
      k_fill_dirs<<<grid_1d(N * (int64_t)K), 256, 0, s>>>(g, cx, cy, K, src.get());
    }
    HBS_LAUNCH_CHECK("k_fill_dirs");
    h.Pdir.alloc((size_t)h.rsel * K);
    std::vector<GemmJob> gj(1);
    gj[0] = {h.VT.get(), src.get(), h.Pdir.get(), h.rsel, K, (int)N, (int)N, (int)N, h.rsel, cmk(1, 0), cmk(0, 0), 0, 0,
             0, 1};
    run_gemms(gj, s);
  }
  HBS_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// Per-Bloch-phase solve
// ---------------------------------------------------------------------------

struct GroupJob {
  cplx alpha;
  int q, nw;                 // angles, Wood's modes
  int rhs_col;               // first column of this group in X / Proj (b's then PW)
  int contour;               // 0 standard, 1 shifted
  const cplx* zp;            // fast path: Z (zr x zc) of the contour
  const cplx* zl;            // plain path: Rows A^{-1} L (zr x 2l), else null
  const cplx* zb;            // plain path: Rows A^{-1} B(alpha) (zr x 2M), else null
  const cplx* sl;            // wall sample rows SL, SR (4S x 2M)
  const cplx* sr;
  const cplx* ck;            // contour nodes (M)
  double wkap[4];            // kappa_n of Wood's modes
  cplx wkn[4];               // k_n of Wood's modes
  int64_t s_off, r_off;      // offsets of S (nS x nS) and rhs (nS x q) in the pools
  int64_t piv_off;
  int nsys;                  // size of the Schur system solved for this group
  // reduced path (compressed periodizer): per-group work arrays
  const cplx* ul;            // U_L, U_R (2M x rC): C_L, C_R rows from the skeleton rows
  const cplx* ur;
  const cplx* vl;            // V_L, V_R (2M x rB): B_L, B_R columns from the skeleton columns
  const cplx* vr;
  cplx* vt;                  // (V_L + alpha V_R)^T  (rB x 2M)
  cplx* qu;                  // Q^{-1} (alpha U_L - alpha^{-2} U_R)  (2M x rC)
  cplx* hm;                  // H = Vt QU  (rB x rC)
  cplx* hc;                  // H [Zc(C rows) | Psel(C rows)]  (rB x (l + rB + q + nw))
  cplx* wd;                  // Wood's: psi^T Wall(alpha) (2M) then w = that QU (rC), per mode
  cplx* qcoef;               // per contour node m: Q's entries qff, qfn, qnf, qnn and 1 / det (5 M)
  cplx* wpsi;                // Wood's sampling weights psi_t(s), s = S..4S-1 (3S per mode)
};

struct Dims {
  int l, M, S, zr;
  double d, omega;
  int64_t ldproj;  // leading dimension of Proj (= zr)
};

// Value of (Rows A^{-1} [column C of the Schur unknowns]) at Rows row r.
__device__ __forceinline__ cplx rows_ainv(const Dims& D, const GroupJob& G, const cplx* proj, int r, int C) {
  const int l = D.l, M = D.M, zr = D.zr;
  if (C < 2 * l) {
    if (G.zl) return G.zl[(int64_t)C * zr + r];
    const int c = C < l ? C : C - l;
    cplx v = G.zp[(int64_t)c * zr + r];
    cplx f = C < l ? cdiv(cmk(1, 0), G.alpha) : G.alpha;
    return cmul(f, v);
  }
  if (C < 2 * l + 2 * M) {
    const int c = C - 2 * l;
    if (G.zb) return G.zb[(int64_t)c * zr + r];
    cplx v = G.zp[(int64_t)(l + c) * zr + r];
    cplx w = G.zp[(int64_t)(l + 2 * M + c) * zr + r];
    return cfma(G.alpha, w, v);
  }
  const int t = C - 2 * l - 2 * M;
  return proj[(int64_t)(G.rhs_col + G.q + t) * D.ldproj + r];
}

// Sampling-row weight psi for Wood's row t at sample row s in [0, 4S): i k_n F_n on
// u(-y0), F_n on u_y(-y0), F_n = e^{-i kappa_n x_s} / S.
__device__ __forceinline__ cplx wood_psi(const Dims& D, const GroupJob& G, int t, int s) {
  const int S = D.S;
  const int kind = s / S, ss = s % S;
  if (kind != 1 && kind != 3) return cmk(0, 0);
  const double xs = -0.5 * D.d + (ss + 0.5) * D.d / S;
  double sn, cs;
  sincos(-G.wkap[t] * xs, &sn, &cs);
  cplx f = cmk(cs / S, sn / S);
  if (kind == 3) return f;
  return cmul(cmul(cmk(0, 1), G.wkn[t]), f);
}

// Schur row functional applied to (Rows A^{-1} column C): row block zeta, xi or Wood's.
__device__ cplx row_functional(const Dims& D, const GroupJob& G, const cplx* proj, int Rw, int C) {
  const int l = D.l, M = D.M, S = D.S;
  if (Rw < 2 * l) return rows_ainv(D, G, proj, Rw, C);
  if (Rw < 2 * l + 2 * M) {
    const int r = Rw - 2 * l;
    cplx a = rows_ainv(D, G, proj, 2 * l + r, C);
    cplx b = rows_ainv(D, G, proj, 2 * l + 2 * M + r, C);
    cplx a2 = cmul(G.alpha, G.alpha);
    return csub(cmul(G.alpha, a), cdiv(b, a2));
  }
  const int t = Rw - 2 * l - 2 * M;
  cplx acc = cmk(0, 0);
  cplx aj = cdiv(cmk(1, 0), G.alpha);
  for (int jj = 0; jj < 3; ++jj) {
    cplx part = cmk(0, 0);
    for (int sidx = S; sidx < 4 * S; ++sidx) {
      cplx p = wood_psi(D, G, t, sidx);
      if (p.x == 0.0 && p.y == 0.0) continue;
      part = cfma(p, rows_ainv(D, G, proj, 2 * l + 4 * M + 4 * S * jj + sidx, C), part);
    }
    acc = cfma(aj, part, acc);
    aj = cmul(aj, G.alpha);
  }
  return acc;
}

__device__ __forceinline__ cplx plane_wave_at(double kap, cplx kn, double x, double y, bool dy) {
  // e^{i kappa x} e^{i k y}, k complex
  cplx e = cexp(cmk(-kn.y * y, kap * x + kn.x * y));
  if (dy) e = cmul(cmul(cmk(0, 1), kn), e);
  return e;
}

__device__ __forceinline__ cplx sample_point_pw(const Dims& D, const GroupJob& G, int t, int r, double y0) {
  const int S = D.S;
  const int kind = r / S, ss = r % S;
  const double xs = -0.5 * D.d + (ss + 0.5) * D.d / S;
  const double ys = (kind == 0 || kind == 2) ? y0 : -y0;
  return plane_wave_at(G.wkap[t], G.wkn[t], xs, ys, kind >= 2);
}

// Assemble S (nS x nS) and the right-hand sides (nS x q) of every group.
__global__ void k_assemble(Dims D, const GroupJob* groups, const cplx* proj, double y0, cplx* Spool, cplx* Rpool) {
  const GroupJob G = groups[blockIdx.y];
  const int l = D.l, M = D.M, S = D.S;
  const int nS = 2 * l + 2 * M + G.nw;
  const int64_t tot = (int64_t)nS * (nS + G.q);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int Rw = (int)(e % nS);
    const int C = (int)(e / nS);
    if (C >= nS) {
      // right-hand side: -(row functional of Rows X_b)
      const int i = C - nS;
      cplx v;
      if (Rw < 2 * l) {
        v = proj[(int64_t)(G.rhs_col + i) * D.ldproj + Rw];
      } else if (Rw < 2 * l + 2 * M) {
        const int r = Rw - 2 * l;
        cplx a = proj[(int64_t)(G.rhs_col + i) * D.ldproj + 2 * l + r];
        cplx b = proj[(int64_t)(G.rhs_col + i) * D.ldproj + 2 * l + 2 * M + r];
        v = csub(cmul(G.alpha, a), cdiv(b, cmul(G.alpha, G.alpha)));
      } else {
        const int t = Rw - 2 * l - 2 * M;
        v = cmk(0, 0);
        cplx aj = cdiv(cmk(1, 0), G.alpha);
        for (int jj = 0; jj < 3; ++jj) {
          cplx part = cmk(0, 0);
          for (int sidx = S; sidx < 4 * S; ++sidx) {
            cplx p = wood_psi(D, G, t, sidx);
            if (p.x == 0.0 && p.y == 0.0) continue;
            part = cfma(p, proj[(int64_t)(G.rhs_col + i) * D.ldproj + 2 * l + 4 * M + 4 * S * jj + sidx], part);
          }
          v = cfma(aj, part, v);
          aj = cmul(aj, G.alpha);
        }
      }
      Rpool[G.r_off + (int64_t)i * nS + Rw] = cmk(-v.x, -v.y);
      continue;
    }
    cplx v = row_functional(D, G, proj, Rw, C);
    v = cmk(-v.x, -v.y);
    if (Rw < 2 * l) {
      if (C == Rw) v.x -= 1.0;
    } else if (Rw < 2 * l + 2 * M) {
      const int r = Rw - 2 * l;
      if (C >= 2 * l && C < 2 * l + 2 * M) {
        const int c = C - 2 * l;
        const int m = r % M, cm = c % M;
        if (m == cm) {
          // Q(alpha) entries (rows [f; fn], columns [mu; nu]) at contour node m
          cplx km = G.ck[m];
          cplx sq = cmul(csqrt_principal(cmk(D.omega - km.x, -km.y)), csqrt_principal(cmk(D.omega + km.x, km.y)));
          cplx ee = cexp(cmk(-sq.y * D.d, sq.x * D.d));
          cplx ia = cdiv(cmk(1, 0), G.alpha);
          cplx ap = cadd(G.alpha, ia), am = csub(G.alpha, ia);
          cplx q;
          const bool frow = r < M, mucol = c < M;
          if (frow && mucol) q = cdiv(cmul(cmul(ee, cmk(0, 1)), am), cscale(sq, 2.0));
          else if (frow && !mucol) q = csub(cmk(1, 0), cscale(cmul(ee, ap), 0.5));
          else if (!frow && mucol) q = cadd(cmk(-1, 0), cscale(cmul(ee, ap), 0.5));
          else q = cscale(cmul(cmul(ee, cmk(0, 1)), cmul(sq, am)), 0.5);
          v = cadd(v, q);
        }
      }
    } else {
      const int t = Rw - 2 * l - 2 * M;
      if (C >= 2 * l && C < 2 * l + 2 * M) {
        // psi^T Wall(alpha) column
        const int c = C - 2 * l;
        cplx acc = cmk(0, 0);
        for (int sidx = S; sidx < 4 * S; ++sidx) {
          cplx p = wood_psi(D, G, t, sidx);
          if (p.x == 0.0 && p.y == 0.0) continue;
          cplx wv = cfma(G.alpha, G.sr[(int64_t)c * 4 * S + sidx], G.sl[(int64_t)c * 4 * S + sidx]);
          acc = cfma(p, wv, acc);
        }
        v = cadd(v, acc);
      } else if (C >= 2 * l + 2 * M) {
        const int t2 = C - 2 * l - 2 * M;
        cplx acc = cmk(0, 0);
        for (int sidx = S; sidx < 4 * S; ++sidx) {
          cplx p = wood_psi(D, G, t, sidx);
          if (p.x == 0.0 && p.y == 0.0) continue;
          acc = cfma(p, sample_point_pw(D, G, t2, sidx, y0), acc);
        }
        v = cadd(v, acc);
      }
    }
    Spool[G.s_off + (int64_t)C * nS + Rw] = v;
  }
}

// Batched dense solve S U = Rhs (Gaussian elimination with partial pivoting on the
// augmented matrix), one CTA per group.  illcond[g] = 1 if a pivot fell below
// 1e-14 times the largest pivot.
template <int NT>
__global__ void __launch_bounds__(NT) k_schur_solve(Dims D, const GroupJob* groups, cplx* Spool, cplx* Rpool,
                                                    int* illcond) {
  // Right-looking LU with partial pivoting of the augmented system [S | R] (one CTA per
  // Bloch group), blocked by panels of NB columns: the panel is factored column by
  // column, U12 = L11^{-1} A12 follows by forward substitution (one thread per column),
  // and the trailing matrix gets one rank-NB update from shared-memory tiles of L21 and
  // U12 with 4 x 4 register tiles per thread.
  constexpr int NB = 16, TM = 64;
  static_assert(NT == 256, "16 x 16 threads per trailing tile");
  __shared__ long long redv[32];
  __shared__ int redi[32];
  __shared__ cplx sh_ip;
  __shared__ cplx Ls[NB][TM + 1];
  __shared__ cplx Us[NB][TM + 1];
  __shared__ cplx L11[NB][NB + 1];
  const GroupJob G = groups[blockIdx.x];
  const int n = G.nsys, q = G.q, nc = n + q;
  cplx* A = Spool + G.s_off;
  cplx* B = Rpool + G.r_off;
  auto col = [&](int j) -> cplx* { return j < n ? A + (int64_t)j * n : B + (int64_t)(j - n) * n; };
  const int tid = threadIdx.x;
  double pmax = 0.0, pmin = 1e300;
  for (int k0 = 0; k0 < n; k0 += NB) {
    const int nb = min(NB, n - k0);
    for (int c = k0; c < k0 + nb; ++c) {
      cplx* ac = A + (int64_t)c * n;
      long long best = kNoKey;
      int bi = 0x7fffffff;
      for (int i = c + tid; i < n; i += NT) {
        const long long v = nkey(cabs2(ac[i]));
        if (better(v, i, best, bi)) { best = v; bi = i; }
      }
      long long kv;
      int p;
      block_argmax_key<NT>(best, bi, redv, redi, &kv, &p);
      if (tid == 0) {  // pivot range for the conditioning flag (read by thread 0)
        const double pv = __longlong_as_double(kv);
        pmax = fmax(pmax, pv);
        pmin = fmin(pmin, pv);
      }
      if (p != c) {
        for (int j = tid; j < nc; j += NT) {
          cplx* cj = col(j);
          const cplx t = cj[c];
          cj[c] = cj[p];
          cj[p] = t;
        }
      }
      __syncthreads();
      if (tid == 0) {
        const cplx dv = ac[c];
        sh_ip = cabs2(dv) > 0.0 ? cdiv(cmk(1, 0), dv) : cmk(0, 0);
      }
      __syncthreads();
      const cplx ip = sh_ip;
      for (int i = c + 1 + tid; i < n; i += NT) ac[i] = cmul(ac[i], ip);
      __syncthreads();
      for (int j = c + 1; j < k0 + nb; ++j) {
        cplx* aj = A + (int64_t)j * n;
        const cplx ucj = aj[c];
        for (int i = c + 1 + tid; i < n; i += NT) aj[i] = cfms(ac[i], ucj, aj[i]);
      }
      __syncthreads();
    }
    const int j0 = k0 + nb;
    if (j0 >= nc) break;
    for (int e = tid; e < NB * NB; e += NT) {
      const int r = e % NB, cc = e / NB;
      L11[r][cc] = (r < nb && cc < nb) ? A[(int64_t)(k0 + cc) * n + k0 + r] : cmk(0, 0);
    }
    __syncthreads();
    for (int j = j0 + tid; j < nc; j += NT) {
      cplx* aj = col(j) + k0;
      cplx u[NB];
#pragma unroll
      for (int r = 0; r < NB; ++r) u[r] = r < nb ? aj[r] : cmk(0, 0);
#pragma unroll
      for (int cc = 0; cc < NB; ++cc)
#pragma unroll
        for (int r = cc + 1; r < NB; ++r) u[r] = cfms(L11[r][cc], u[cc], u[r]);
#pragma unroll
      for (int r = 0; r < NB; ++r)
        if (r < nb) aj[r] = u[r];
    }
    __syncthreads();
    const int rows = n - j0, cols = nc - j0;
    const int tr = tid & 15, tc = tid >> 4;
    for (int rt = 0; rt < rows; rt += TM) {
      for (int ct = 0; ct < cols; ct += TM) {
        for (int e = tid; e < TM * NB; e += NT) {
          const int r = e % TM, kk = e / TM;
          const int i = j0 + rt + r;
          Ls[kk][r] = (i < n && kk < nb) ? A[(int64_t)(k0 + kk) * n + i] : cmk(0, 0);
        }
        for (int e = tid; e < TM * NB; e += NT) {
          const int kk = e % NB, c = e / NB;
          const int j = j0 + ct + c;
          Us[kk][c] = (j < nc && kk < nb) ? col(j)[k0 + kk] : cmk(0, 0);
        }
        __syncthreads();
        cplx acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = cmk(0, 0);
        for (int kk = 0; kk < nb; ++kk) {
          cplx la[4], ub[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) la[a] = Ls[kk][tr + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) ub[b] = Us[kk][tc + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = cfma(la[a], ub[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int j = j0 + ct + tc + 16 * b;
          if (j >= nc) continue;
          cplx* cj = col(j);
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = j0 + rt + tr + 16 * a;
            if (i < n) cj[i] = csub(cj[i], acc[a][b]);
          }
        }
        __syncthreads();
      }
    }
  }
  // back substitution, one RHS per warp
  const int lane = tid & 31, warp = tid >> 5;
  for (int j = warp; j < q; j += NT / 32) {
    cplx* b = B + (int64_t)j * n;
    for (int i = n - 1; i >= 0; --i) {
      cplx acc = cmk(0, 0);
      for (int t = i + 1 + lane; t < n; t += 32) acc = cfma(A[(int64_t)t * n + i], b[t], acc);
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) b[i] = cdiv(csub(b[i], acc), A[(int64_t)i * n + i]);
      __syncwarp();
    }
  }
  if (tid == 0) illcond[blockIdx.x] = (pmin <= 1e-28 * pmax) ? 1 : 0;
}

// The same blocked LU on CL CTAs per Bloch group (a cooperative launch over all groups):
// CTA 0 of the group factors each panel while the others wait at a grid barrier, then all
// CL CTAs share the U12 columns and the trailing-update tiles, and the back substitution's
// right-hand sides.  Three bounded grid barriers per panel (all groups advance together;
// `npan` is the largest panel count).  Used when the groups are fewer than the SMs, so
// that every SM takes part.
// Element arithmetic of the Schur LU for complex FP64 (cplx) and complex double-float (dfc).
__device__ __forceinline__ long long lu_key(const cplx& v) { return nkey(cabs2(v)); }
__device__ __forceinline__ long long lu_key(const dfc& v) {
  return (long long)__float_as_uint(fmaf(v.rh, v.rh, v.ih * v.ih));  // |v|^2 to float precision
}
__device__ __forceinline__ bool lu_key_nonzero(long long k, const cplx*) { return __longlong_as_double(k) > 0.0; }
__device__ __forceinline__ bool lu_key_nonzero(long long k, const dfc*) { return __uint_as_float((unsigned)k) > 0.f; }
__device__ __forceinline__ double lu_key_value(long long k, const cplx*) { return __longlong_as_double(k); }
__device__ __forceinline__ double lu_key_value(long long k, const dfc*) { return (double)__uint_as_float((unsigned)k); }
__device__ __forceinline__ cplx lu_recip(const cplx& d) { return cabs2(d) > 0.0 ? cdiv(cmk(1, 0), d) : cmk(0, 0); }
__device__ __forceinline__ dfc lu_recip(const dfc& d) { return dfc_recip(d); }
__device__ __forceinline__ cplx lu_mul(const cplx& a, const cplx& b) { return cmul(a, b); }
__device__ __forceinline__ dfc lu_mul(const dfc& a, const dfc& b) { return dfc_mul(a, b); }
// c - a b
__device__ __forceinline__ cplx lu_fms(const cplx& a, const cplx& b, const cplx& c) { return cfms(a, b, c); }
__device__ __forceinline__ dfc lu_fms(const dfc& a, const dfc& b, const dfc& c) {
  dfc r = c;
  dfc_sub_mul(a, b, r);
  return r;
}
// acc += a b (lazy for dfc; lu_norm finishes it)
__device__ __forceinline__ void lu_acc(const cplx& a, const cplx& b, cplx& acc) { acc = cfma(a, b, acc); }
__device__ __forceinline__ void lu_acc(const dfc& a, const dfc& b, dfc& acc) {
  df_mac(a.rh, a.rl, b.rh, b.rl, acc.rh, acc.rl);
  df_mac(-a.ih, -a.il, b.ih, b.il, acc.rh, acc.rl);
  df_mac(a.rh, a.rl, b.ih, b.il, acc.ih, acc.il);
  df_mac(a.ih, a.il, b.rh, b.rl, acc.ih, acc.il);
}
__device__ __forceinline__ void lu_norm(cplx&) {}
__device__ __forceinline__ void lu_norm(dfc& a) { dfc_norm(a); }
__device__ __forceinline__ cplx lu_sub(const cplx& c, const cplx& a) { return csub(c, a); }
__device__ __forceinline__ dfc lu_sub(const dfc& c, const dfc& a) {
  dfc r = c;
  df_add_to(-a.rh, -a.rl, r.rh, r.rl);
  df_add_to(-a.ih, -a.il, r.ih, r.il);
  dfc_norm(r);
  return r;
}
template <typename T> __device__ __forceinline__ T lu_zero();
template <> __device__ __forceinline__ cplx lu_zero<cplx>() { return cmk(0, 0); }
template <> __device__ __forceinline__ dfc lu_zero<dfc>() { return {0.f, 0.f, 0.f, 0.f}; }
// warp sum (result in every lane)
__device__ __forceinline__ cplx lu_warp_sum(cplx a) {
  for (int o = 16; o > 0; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
    a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
  }
  return a;
}
__device__ __forceinline__ dfc lu_warp_sum(dfc a) { return dfc_warp_sum(a); }

// CL CTAs per Bloch group factor [S | R] with the panel-blocked LU of k_schur_solve: the
// panel by CTA 0 of the group, U12 and the trailing update split over the group's CTAs,
// three grid barriers per panel (every wait bounded).  The row interchanges are recorded
// in pivpool (pstride per group) for a later refinement.  DF: the arithmetic is double-float on
// the FP32 pipes, with [S | R] held in place as float pairs between a conversion pass at
// the start and one at the end (pivots chosen on |a|^2 to float precision); the caller
// then refines the solution once against the FP64 system.
template <int NT, bool DF>
__global__ void __launch_bounds__(NT) k_schur_coop(Dims D, const GroupJob* groups, int ng, int CL, int npan,
                                                   cplx* Spool, cplx* Rpool, int* illcond, int* pivpool,
                                                   int pstride, GridSync* gs) {
  using T = typename std::conditional<DF, dfc, cplx>::type;
  constexpr int NB = 16, TM = 64;
  static_assert(NT == 256, "16 x 16 threads per trailing tile");
  __shared__ long long redv[32];
  __shared__ int redi[32];
  __shared__ T sh_ip;
  __shared__ T Ls[NB][TM + 1];
  __shared__ T Us[NB][TM + 1];
  __shared__ T L11[NB][NB + 1];
  const int g = blockIdx.x / CL, rank = blockIdx.x % CL;
  const bool act = g < ng;
  int n = 0, q = 0;
  cplx* A64 = nullptr;
  cplx* B64 = nullptr;
  int* piv = nullptr;
  if (act) {
    const GroupJob G = groups[g];
    n = G.nsys;
    q = G.q;
    A64 = Spool + G.s_off;
    B64 = Rpool + G.r_off;
    piv = pivpool + (int64_t)g * pstride;
  }
  T* A = reinterpret_cast<T*>(A64);
  T* B = reinterpret_cast<T*>(B64);
  const int nc = n + q;
  auto col = [&](int j) -> T* { return j < n ? A + (int64_t)j * n : B + (int64_t)(j - n) * n; };
  auto col64 = [&](int j) -> cplx* { return j < n ? A64 + (int64_t)j * n : B64 + (int64_t)(j - n) * n; };
  const int tid = threadIdx.x;
  if constexpr (DF) {
    if (act)
      for (int j = rank; j < nc; j += CL) {
        cplx* c64 = col64(j);
        dfc* cd = reinterpret_cast<dfc*>(c64);
        for (int i = tid; i < n; i += NT) cd[i] = to_dfc_bits(c64[i]);
      }
    if (grid_sync(gs) < 0) return;
  }
  double pmax = 0.0, pmin = 1e300;
  for (int pn = 0; pn < npan; ++pn) {
    const int k0 = pn * NB;
    const bool live = act && k0 < n;
    const int nb = live ? min(NB, n - k0) : 0;
    if (live && rank == 0) {
      for (int c = k0; c < k0 + nb; ++c) {
        T* ac = A + (int64_t)c * n;
        long long best = kNoKey;
        int bi = 0x7fffffff;
        for (int i = c + tid; i < n; i += NT) {
          const long long v = lu_key(ac[i]);
          if (better(v, i, best, bi)) { best = v; bi = i; }
        }
        long long kv;
        int p;
        block_argmax_key<NT>(best, bi, redv, redi, &kv, &p);
        if (tid == 0) {  // pivot range for the conditioning flag (read by thread 0)
          const double pv = lu_key_value(kv, A);
          pmax = fmax(pmax, pv);
          pmin = fmin(pmin, pv);
          piv[c] = p;
        }
        if (p != c) {
          for (int j = tid; j < nc; j += NT) {
            T* cj = col(j);
            const T t = cj[c];
            cj[c] = cj[p];
            cj[p] = t;
          }
        }
        __syncthreads();
        if (tid == 0) sh_ip = lu_recip(ac[c]);
        __syncthreads();
        const T ip = sh_ip;
        for (int i = c + 1 + tid; i < n; i += NT) ac[i] = lu_mul(ac[i], ip);
        __syncthreads();
        for (int j = c + 1; j < k0 + nb; ++j) {
          T* aj = A + (int64_t)j * n;
          const T ucj = aj[c];
          for (int i = c + 1 + tid; i < n; i += NT) aj[i] = lu_fms(ac[i], ucj, aj[i]);
        }
        __syncthreads();
      }
    }
    if (grid_sync(gs) < 0) return;
    const int j0 = k0 + nb;
    const bool upd = live && j0 < nc;
    if (upd) {
      for (int e = tid; e < NB * NB; e += NT) {
        const int r = e % NB, cc = e / NB;
        L11[r][cc] = (r < nb && cc < nb) ? A[(int64_t)(k0 + cc) * n + k0 + r] : lu_zero<T>();
      }
      __syncthreads();
      for (int j = j0 + rank * NT + tid; j < nc; j += CL * NT) {
        T* aj = col(j) + k0;
        T u[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) u[r] = r < nb ? aj[r] : lu_zero<T>();
#pragma unroll
        for (int cc = 0; cc < NB; ++cc)
#pragma unroll
          for (int r = cc + 1; r < NB; ++r) u[r] = lu_fms(L11[r][cc], u[cc], u[r]);
#pragma unroll
        for (int r = 0; r < NB; ++r)
          if (r < nb) aj[r] = u[r];
      }
    }
    if (grid_sync(gs) < 0) return;
    if (upd) {
      const int rows = n - j0, cols = nc - j0;
      const int nrt = (rows + TM - 1) / TM, nct = (cols + TM - 1) / TM;
      const int tr = tid & 15, tc = tid >> 4;
      for (int tt = rank; tt < nrt * nct; tt += CL) {
        const int rt = (tt % nrt) * TM, ct = (tt / nrt) * TM;
        for (int e = tid; e < TM * NB; e += NT) {
          const int r = e % TM, kk = e / TM;
          const int i = j0 + rt + r;
          Ls[kk][r] = (i < n && kk < nb) ? A[(int64_t)(k0 + kk) * n + i] : lu_zero<T>();
        }
        for (int e = tid; e < TM * NB; e += NT) {
          const int kk = e % NB, c = e / NB;
          const int j = j0 + ct + c;
          Us[kk][c] = (j < nc && kk < nb) ? col(j)[k0 + kk] : lu_zero<T>();
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = lu_zero<T>();
        for (int kk = 0; kk < nb; ++kk) {
          T la[4], ub[4];
#pragma unroll
          for (int a = 0; a < 4; ++a) la[a] = Ls[kk][tr + 16 * a];
#pragma unroll
          for (int b = 0; b < 4; ++b) ub[b] = Us[kk][tc + 16 * b];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) lu_acc(la[a], ub[b], acc[a][b]);
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int j = j0 + ct + tc + 16 * b;
          if (j >= nc) continue;
          T* cj = col(j);
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = j0 + rt + tr + 16 * a;
            if (i < n) {
              lu_norm(acc[a][b]);
              cj[i] = lu_sub(cj[i], acc[a][b]);
            }
          }
        }
        __syncthreads();
      }
    }
    if (grid_sync(gs) < 0) return;
  }
  if (act) {
    // back substitution, one right-hand side per warp of the group's CTAs
    const int lane = tid & 31, warp = tid >> 5;
    for (int j = rank * (NT / 32) + warp; j < q; j += CL * (NT / 32)) {
      T* b = B + (int64_t)j * n;
      for (int i = n - 1; i >= 0; --i) {
        T acc = lu_zero<T>();
        for (int t = i + 1 + lane; t < n; t += 32) lu_acc(A[(int64_t)t * n + i], b[t], acc);
        acc = lu_warp_sum(acc);
        if (lane == 0) b[i] = lu_mul(lu_sub(b[i], acc), lu_recip(A[(int64_t)i * n + i]));
        __syncwarp();
      }
    }
    if (rank == 0 && tid == 0) illcond[g] = (pmin <= 1e-28 * pmax) ? 1 : 0;
  }
  if constexpr (DF) {
    if (grid_sync(gs) < 0) return;  // every CTA of the group is done with [S | R]
    if (act)
      for (int j = rank; j < nc; j += CL) {
        cplx* c64 = col64(j);
        const dfc* cd = reinterpret_cast<const dfc*>(c64);
        for (int i = tid; i < n; i += NT) c64[i] = from_dfc_bits(cd[i]);  // same 16-byte slot
      }
  }
}

// One step of iterative refinement per group against the FP64 system (after a factorization
// in double-float): Rres holds R - S X (computed in FP64); solve (LU) d = P Rres with the
// stored factors and pivots, and X += d.  One single-warp CTA per group and right-hand side
// (CTA g qmax + j: right-hand side j of group g), in shared memory: the triangular solves are
// sequential in the row index, so the parallelism is across the right-hand sides of all
// groups.
__global__ void __launch_bounds__(32) k_schur_refine(const GroupJob* groups, const cplx* Spool, cplx* Rpool,
                                                     const cplx* Rres, const int* pivpool, int pstride, int qmax) {
  extern __shared__ cplx sref[];  // n (1/U_ii) + n (the right-hand side)
  const int g = (int)(blockIdx.x / (unsigned)qmax), j = (int)(blockIdx.x % (unsigned)qmax);
  const GroupJob G = groups[g];
  const int n = G.nsys;
  if (j >= G.q) return;
  const cplx* A = Spool + G.s_off;
  const int* piv = pivpool + (int64_t)g * pstride;
  const int lane = threadIdx.x;
  cplx* inv = sref;
  cplx* r = sref + n;
  const cplx* rr = Rres + G.r_off + (int64_t)j * n;
  for (int i = lane; i < n; i += 32) {
    inv[i] = cdiv(cmk(1, 0), A[(int64_t)i * n + i]);
    r[i] = rr[i];
  }
  __syncwarp();
  if (lane == 0)
    for (int c = 0; c < n; ++c) {
      const int p = piv[c];
      if (p != c) {
        const cplx t = r[c];
        r[c] = r[p];
        r[p] = t;
      }
    }
  __syncwarp();
  for (int t = 0; t < n; ++t) {  // unit lower L
    const cplx rt = r[t];
    __syncwarp();
    for (int i = t + 1 + lane; i < n; i += 32) r[i] = cfms(A[(int64_t)t * n + i], rt, r[i]);
    __syncwarp();
  }
  for (int t = n - 1; t >= 0; --t) {  // upper U
    if (lane == 0) r[t] = cmul(r[t], inv[t]);
    __syncwarp();
    const cplx rt = r[t];
    for (int i = lane; i < t; i += 32) r[i] = cfms(A[(int64_t)t * n + i], rt, r[i]);
    __syncwarp();
  }
  cplx* x = Rpool + G.r_off + (int64_t)j * n;
  for (int i = lane; i < n; i += 32) x[i] = cadd(x[i], r[i]);
}

// Factor and solve every group's Schur system: CL CTAs per group in one cooperative launch
// when the groups leave SMs idle, else one CTA per group.  In the thread's double-float
// mode the cooperative factorization runs in double-float and the solution is refined once
// against the FP64 system (residual by an FP64 product, correction with the same factors).
static void schur_solve(const Dims& D, const std::vector<GroupJob>& gjobs, const GroupJob* dg, cplx* Sp, cplx* Rp,
                        int* ill, cudaStream_t s) {
  const int ng = (int)gjobs.size();
  const bool df = gemm_double_float();
  // SM count and residency of the variant this call launches, per device (looked up once
  // per device and variant under a lock: solves may run concurrently)
  int sms = 0, per_sm = 0;
  {
    static std::mutex mu;
    static std::map<std::pair<int, bool>, std::pair<int, int>> occ;
    int dev = 0;
    HBS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ.find({dev, df});
    if (it == occ.end()) {
      int sm = 0, per = 0;
      HBS_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
      if (df) HBS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_schur_coop<256, true>, 256, 0));
      else HBS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_schur_coop<256, false>, 256, 0));
      it = occ.emplace(std::make_pair(dev, df), std::make_pair(sm, per)).first;
    }
    sms = it->second.first;
    per_sm = it->second.second;
  }
  // every CTA of the cooperative launch must be co-resident: ng * CL <= sms * per_sm
  const int cl_max = std::min(4, (sms * std::min(per_sm, 2)) / std::max(ng, 1));
  if (cl_max < 2) {
    k_schur_solve<256><<<ng, 256, 0, s>>>(D, dg, Sp, Rp, ill);
    return;
  }
  int nmax = 0;
  int64_t send = 0, rend = 0;
  for (const auto& G : gjobs) {
    nmax = std::max(nmax, G.nsys);
    send = std::max<int64_t>(send, G.s_off + (int64_t)G.nsys * G.nsys);
    rend = std::max<int64_t>(rend, G.r_off + (int64_t)G.nsys * G.q);
  }
  // CTAs per group: 2, 3 or 4 (tuned per shape class when autotuning is on; the most that
  // stay co-resident by default)
  int n_pow = 1, g_pow = 1;
  while (n_pow < nmax) n_pow *= 2;
  while (g_pow < ng) g_pow *= 2;
  const std::string tkey = "schur/n" + std::to_string(n_pow) + "/g" + std::to_string(g_pow) + (df ? "/df" : "");
  int var = tune::choose(tkey, 3, cl_max - 2);
  if (var + 2 > cl_max) {  // more CTAs than stay co-resident: not a candidate
    if (tune::exploring(tkey, 3)) tune::record(tkey, var, 3, 1e30f);
    var = cl_max - 2;
  }
  const int CL = var + 2;
  tune::Timed timed(tkey, var, 3, s);
  const int npan = (nmax + 15) / 16;
  DevBuf<GridSync> gs(1);
  DevBuf<int> piv((size_t)ng * std::max(nmax, 1));
  DevBuf<cplx> S0, R0;
  if (df) {  // the FP64 system, for the refinement
    S0.alloc(std::max<int64_t>(send, 1));
    R0.alloc(std::max<int64_t>(rend, 1));
    HBS_CUDA(cudaMemcpyAsync(S0.get(), Sp, sizeof(cplx) * send, cudaMemcpyDeviceToDevice, s));
    HBS_CUDA(cudaMemcpyAsync(R0.get(), Rp, sizeof(cplx) * rend, cudaMemcpyDeviceToDevice, s));
  }
  HBS_CUDA(cudaMemsetAsync(gs.get(), 0, sizeof(GridSync), s));
  Dims a0 = D;
  const GroupJob* a1 = dg;
  int a2 = ng, a3 = CL, a4 = npan;
  cplx* a5 = Sp;
  cplx* a6 = Rp;
  int* a7 = ill;
  int* a8 = piv.get();
  int a9 = nmax;
  GridSync* a10 = gs.get();
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10};
  {
    std::lock_guard<std::mutex> lock(coop_mutex());
    const void* fn = df ? (const void*)k_schur_coop<256, true> : (const void*)k_schur_coop<256, false>;
    HBS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(ng * CL), dim3(256), args, 0, s));
    GridSync hg{};
    read_to_host(&hg, gs.get(), sizeof(GridSync), s);
    if (hg.timed_out) throw Error(HBS_ERR_TIMEOUT, "Schur factorization: a grid barrier wait gave up");
  }
  if (!df) return;
  // R0 <- R0 - S0 X (FP64), then X += (LU)^{-1} P R0
  {
    GemmModeScope fp64(HBS_PRECISION_FP64);
    std::vector<GemmJob> gj;
    for (const auto& G : gjobs)
      gj.push_back({S0.get() + G.s_off, Rp + G.r_off, R0.get() + G.r_off, G.nsys, G.q, G.nsys, G.nsys, G.nsys,
                    G.nsys, cmk(-1, 0), cmk(1, 0), 0, 0, 0});
    run_gemms(gj, s);
  }
  {
    prof::KScope _ks("k_schur_refine", s);
    const size_t shm = (size_t)2 * nmax * sizeof(cplx);
    HBS_CUDA(raise_smem_limit((const void*)k_schur_refine, shm));
    int qmax = 1;
    for (const auto& G : gjobs) qmax = std::max(qmax, G.q);
    k_schur_refine<<<(unsigned)(ng * qmax), 32, shm, s>>>(dg, Sp, Rp, R0.get(), piv.get(), nmax, qmax);
  }
  HBS_LAUNCH_CHECK("k_schur_refine");
}

struct AngleJob {
  int group;
  int col;            // index of this angle within its group
  double kappa;       // kappa^i = w cos(theta)
  double k0;          // w |sin theta|
  int n_min, n_max;
  int64_t out_off;    // into c/d output arrays
};

// Bragg amplitudes and flux per angle: samples of u at +-y0 from
// sum_j alpha^j E_j eta + Wall(alpha) xi + PW a, with
// E_j eta = Proj[E_j, b] - (Rows A^{-1} [L B PW]) [zeta; xi; a], then the DFT.
__global__ void k_bragg(Dims D, const GroupJob* groups, const AngleJob* angles, const cplx* proj, const cplx* Rpool,
                        double y0, cplx* cout, cplx* dout, double* flux) {
  extern __shared__ cplx samp[];  // 2S
  const AngleJob A = angles[blockIdx.x];
  const GroupJob G = groups[A.group];
  const int l = D.l, M = D.M, S = D.S;
  const int nS = 2 * l + 2 * M + G.nw;
  const cplx* u = Rpool + G.r_off + (int64_t)A.col * nS;
  for (int r = threadIdx.x; r < 2 * S; r += blockDim.x) {
    cplx acc = cmk(0, 0);
    cplx aj = cdiv(cmk(1, 0), G.alpha);
    for (int jj = 0; jj < 3; ++jj) {
      const int row = 2 * l + 4 * M + 4 * S * jj + r;
      cplx part = proj[(int64_t)(G.rhs_col + A.col) * D.ldproj + row];
      for (int C = 0; C < nS; ++C) part = csub(part, cmul(rows_ainv(D, G, proj, row, C), u[C]));
      acc = cfma(aj, part, acc);
      aj = cmul(aj, G.alpha);
    }
    for (int c = 0; c < 2 * M; ++c) {
      cplx wv = cfma(G.alpha, G.sr[(int64_t)c * 4 * S + r], G.sl[(int64_t)c * 4 * S + r]);
      acc = cfma(wv, u[2 * l + c], acc);
    }
    for (int t = 0; t < G.nw; ++t) acc = cfma(sample_point_pw(D, G, t, r, y0), u[2 * l + 2 * M + t], acc);
    samp[r] = acc;
  }
  __syncthreads();
  __shared__ double fl[32];
  const int no = A.n_max - A.n_min + 1;
  double fsum = 0.0;
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    const int n = A.n_min + o;
    const double kap = A.kappa + 2.0 * HBS_PI * n / D.d;
    cplx cn = cmk(0, 0), dn = cmk(0, 0);
    for (int s = 0; s < S; ++s) {
      const double xs = -0.5 * D.d + (s + 0.5) * D.d / S;
      double sn, cs;
      sincos(-kap * xs, &sn, &cs);
      cplx e = cmk(cs / S, sn / S);
      cn = cfma(e, samp[s], cn);
      dn = cfma(e, samp[S + s], dn);
    }
    cout[A.out_off + o] = cn;
    dout[A.out_off + o] = dn;
    const double kn2 = D.omega * D.omega - kap * kap;
    const double kn = kn2 > 0 ? sqrt(kn2) : 0.0;
    cplx dd = dn;
    if (n == 0) {
      double sn, cs;
      sincos(A.k0 * y0, &sn, &cs);
      dd = cadd(dd, cmk(cs, sn));
    }
    fsum += (kn / A.k0) * (cabs2(cn) + cabs2(dd));
  }
  for (int o = 16; o > 0; o >>= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
  if ((threadIdx.x & 31) == 0) fl[threadIdx.x >> 5] = fsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += fl[w];
    flux[blockIdx.x] = fabs(t - 1.0);
  }
}

// Right-hand sides: column c of X gets -e^{i(kappa x + ky y)} (incident data b = -u^i)
// or a Wood's plane wave e^{i(kappa_n x + k_n y)}.
struct RhsCol {
  double kap;
  cplx ky;
  double sign;
};
__global__ void k_fill_rhs(DevGeom g, const RhsCol* cols, int ncol, cplx* X) {
  const int64_t tot = g.n * (int64_t)ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % g.n;
    const int c = (int)(e / g.n);
    const RhsCol rc = cols[c];
    cplx v = cexp(cmk(-rc.ky.y * g.y[i], rc.kap * g.x[i] + rc.ky.x * g.y[i]));
    if (g.comps == 2 && !(i & 1)) {  // transmission sigma row: -(d/dn) / w = -i (kappa n_x + k_y n_y) / w
      const cplx a = cscale(cadd(cmk(rc.kap * g.nx[i], 0.0), cscale(rc.ky, g.ny[i])), 1.0 / g.omega);
      v = cmul(cmk(a.y, -a.x), v);
    }
    X[e] = cscale(v, rc.sign);
  }
}

// columns c0.. of X: s * P (P: N x l)
// Weights of exact trigonometric interpolation in the incidence direction: column c of the
// K x ncol output holds phase_c D_K(psi_c - 2 pi k / K), k = 0..K-1, with D_K the
// interpolation kernel of K equispaced points, D_K(t) = (sin((K - 1) t / 2) / sin(t / 2)
// + cos(K t / 2)) / K (1 at t = 0).  A column with phase 0 (an evanescent plane wave, formed
// directly) gets zeros.
__global__ void k_interp_dirs(const double* psi, const cplx* phase, int64_t ncol, int K, cplx* out) {
  const int64_t tot = ncol * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / K;
    const int k = (int)(e - c * K);
    const cplx ph = phase[c];
    double dk = 0.0;
    if (ph.x != 0.0 || ph.y != 0.0) {
      const double t = psi[c] - 2.0 * HBS_PI * k / K;
      const double sh = sin(0.5 * t);
      dk = fabs(sh) < 1e-12 ? 1.0 : (sin(0.5 * (K - 1) * t) / sh + cos(0.5 * K * t)) / K;
    }
    out[e] = cmk(ph.x * dk, ph.y * dk);
  }
}

__global__ void k_scaled_copy(const cplx* src, int64_t n, cplx f, cplx* dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = cmul(f, src[e]);
}

// ---------------------------------------------------------------------------
// Reduced Schur systems (precomputed path).  With the compressed periodizer,
// C~ = U(alpha) C_sel and B = Y_sel V(alpha)^T with U = alpha U_L - alpha^{-2} U_R and
// V = V_L + alpha V_R (interpolation matrices of the IDs).  The wall rows then read
// Q xi = U gamma with gamma = C_sel A^{-1} (L zeta + Y_sel beta + PW a - b) and beta = V^T xi,
// so xi = Q^{-1} U gamma (Q is 2 x 2 block diagonal) and beta = H gamma, H = V^T Q^{-1} U.
// The unknowns become (zeta, beta, a): 2l + rB + n_wood instead of 2l + 2M + n_wood.
// ---------------------------------------------------------------------------

// Dense interpolation matrix (nout x r) from a recipe: row j = e_{rec.y - off} (kind 0)
// or T[:, rec.y]^T (kind tkind); other kinds give zero rows.
__global__ void k_dense_from_recipe(const int2* rec, int nout, int tkind, const cplx* T, int r, int off, cplx* out) {
  const int64_t tot = (int64_t)nout * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % nout), i = (int)(e / nout);
    const int2 rc = rec[j];
    cplx v = cmk(0, 0);
    if (rc.x == 0) v = cmk(i == rc.y - off ? 1.0 : 0.0, 0.0);
    else if (rc.x == tkind) v = T[i + (int64_t)rc.y * r];
    out[j + (int64_t)i * nout] = v;
  }
}

struct RedDims {
  int l, M, S, rB, rC, rsel;
  double d, omega;
};

__device__ __forceinline__ void q_node(double omega, double d, cplx alpha, cplx km, cplx* qff, cplx* qfn, cplx* qnf,
                                       cplx* qnn) {
  // Q at one contour node: rows [f; fn], columns [mu; nu] (derived from (urep), (f), (fn))
  cplx sq = cmul(csqrt_principal(cmk(omega - km.x, -km.y)), csqrt_principal(cmk(omega + km.x, km.y)));
  cplx ee = cexp(cmk(-sq.y * d, sq.x * d));
  cplx ia = cdiv(cmk(1, 0), alpha);
  cplx ap = cadd(alpha, ia), am = csub(alpha, ia);
  *qff = cdiv(cmul(cmul(ee, cmk(0, 1)), am), cscale(sq, 2.0));
  *qfn = csub(cmk(1, 0), cscale(cmul(ee, ap), 0.5));
  *qnf = cadd(cmk(-1, 0), cscale(cmul(ee, ap), 0.5));
  *qnn = cscale(cmul(cmul(ee, cmk(0, 1)), cmul(sq, am)), 0.5);
}

// Per group, the factors the reduced kernels use many times over: Q's 2 x 2 block of each
// contour node (its four entries and the reciprocal of its determinant) and the Wood's
// sampling weights psi_t(s) of each Wood's mode.
__global__ void k_red_tables(RedDims D, Dims DD, const GroupJob* groups) {
  const GroupJob G = groups[blockIdx.y];
  const int M = D.M, S3 = 3 * D.S;
  const int64_t tot = M + (int64_t)G.nw * S3;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < M) {
      const int m = (int)e;
      cplx qff, qfn, qnf, qnn;
      q_node(D.omega, D.d, G.alpha, G.ck[m], &qff, &qfn, &qnf, &qnn);
      cplx* c = G.qcoef + 5 * (int64_t)m;
      c[0] = qff;
      c[1] = qfn;
      c[2] = qnf;
      c[3] = qnn;
      c[4] = cdiv(cmk(1, 0), csub(cmul(qff, qnn), cmul(qfn, qnf)));
    } else {
      const int64_t q = e - M;
      const int t = (int)(q / S3), sidx = (int)(q % S3);
      G.wpsi[q] = wood_psi(DD, G, t, D.S + sidx);
    }
  }
}

// psi_t(s) for s in [S, 4S) from the group's table.
__device__ __forceinline__ cplx wood_psi_tab(const GroupJob& G, int S, int t, int sidx) {
  return G.wpsi[(int64_t)t * 3 * S + (sidx - S)];
}

// Per group: vt = (V_L + alpha V_R)^T and qu = Q^{-1} (alpha U_L - alpha^{-2} U_R).
__global__ void k_red_prep(RedDims D, const GroupJob* groups) {
  const GroupJob G = groups[blockIdx.y];
  const int M = D.M, M2 = 2 * D.M;
  const int64_t nv = (int64_t)D.rB * M2, nq = (int64_t)M * D.rC;
  const cplx ia2 = cdiv(cmk(1, 0), cmul(G.alpha, G.alpha));
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nv + nq; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nv) {
      const int i = (int)(e % D.rB), mm = (int)(e / D.rB);
      G.vt[i + (int64_t)mm * D.rB] = cfma(G.alpha, G.vr[mm + (int64_t)i * M2], G.vl[mm + (int64_t)i * M2]);
    } else {
      const int64_t q = e - nv;
      const int m = (int)(q % M), c = (int)(q / M);
      const cplx* qc = G.qcoef + 5 * (int64_t)m;
      const cplx qff = qc[0], qfn = qc[1], qnf = qc[2], qnn = qc[3], idet = qc[4];
      const int64_t o = (int64_t)c * M2;
      cplx uf = csub(cmul(G.alpha, G.ul[m + o]), cmul(ia2, G.ur[m + o]));
      cplx un = csub(cmul(G.alpha, G.ul[M + m + o]), cmul(ia2, G.ur[M + m + o]));
      G.qu[m + o] = cmul(csub(cmul(qnn, uf), cmul(qfn, un)), idet);
      G.qu[M + m + o] = cmul(csub(cmul(qff, un), cmul(qnf, uf)), idet);
    }
  }
}

// Wood's rows of one group: wd[t] = [psi_t^T Wall(alpha) (2M) | that times qu (rC)].
__global__ void k_red_wood(RedDims D, const GroupJob* groups, Dims DD) {
  const GroupJob G = groups[blockIdx.x];
  if (G.nw == 0) return;
  const int M2 = 2 * D.M, S4 = 4 * D.S;
  for (int t = 0; t < G.nw; ++t) {
    cplx* w = G.wd + (int64_t)t * (M2 + D.rC);
    for (int mm = threadIdx.x; mm < M2; mm += blockDim.x) {
      cplx acc = cmk(0, 0);
      for (int sidx = D.S; sidx < S4; ++sidx) {
        cplx p = wood_psi_tab(G, D.S, t, sidx);
        if (p.x == 0.0 && p.y == 0.0) continue;
        acc = cfma(p, cfma(G.alpha, G.sr[(int64_t)mm * S4 + sidx], G.sl[(int64_t)mm * S4 + sidx]), acc);
      }
      w[mm] = acc;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < D.rC; c += blockDim.x) {
      cplx acc = cmk(0, 0);
      for (int mm = 0; mm < M2; ++mm) acc = cfma(w[mm], G.qu[mm + (int64_t)c * M2], acc);
      w[M2 + c] = acc;
    }
    __syncthreads();
  }
}

// phi_t . X: Wood's sampling functional over the three images' E rows (ld 12S column X).
__device__ __forceinline__ cplx wood_phi(const Dims& DD, const GroupJob& G, int t, const cplx* X) {
  const int S = DD.S;
  cplx acc = cmk(0, 0);
  cplx aj = cdiv(cmk(1, 0), G.alpha);
  for (int jj = 0; jj < 3; ++jj) {
    cplx part = cmk(0, 0);
    for (int sidx = S; sidx < 4 * S; ++sidx) {
      cplx p = wood_psi_tab(G, S, t, sidx);
      if (p.x == 0.0 && p.y == 0.0) continue;
      part = cfma(p, X[4 * S * jj + sidx], part);
    }
    acc = cfma(aj, part, acc);
    aj = cmul(aj, G.alpha);
  }
  return acc;
}

__global__ void k_red_assemble(RedDims D, Dims DD, const GroupJob* groups, const cplx* Zc, const cplx* Psel,
                               const cplx* EZ, const cplx* EP, double y0, cplx* Spool, cplx* Rpool) {
  const GroupJob G = groups[blockIdx.y];
  const int l = D.l, rB = D.rB, rC = D.rC, rsel = D.rsel, S12 = 12 * D.S;
  const int n = G.nsys, M2 = 2 * D.M;
  const cplx ia = cdiv(cmk(1, 0), G.alpha);
  const int64_t tot = (int64_t)n * (n + G.q);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n);
    const int C = (int)(e / n);
    // column description
    int kind, idx;  // 0 zeta (base col idx, factor f), 1 beta (idx), 2 Wood (idx), 3 rhs (idx)
    cplx f = cmk(1, 0);
    if (C >= n) { kind = 3; idx = C - n; }
    else if (C < 2 * l) { kind = 0; idx = C < l ? C : C - l; f = C < l ? ia : G.alpha; }
    else if (C < 2 * l + rB) { kind = 1; idx = C - 2 * l; }
    else { kind = 2; idx = C - 2 * l - rB; }
    // Zc / Psel column for this unknown
    const int zcol = kind == 0 ? idx : (kind == 1 ? l + idx : -1);
    const int pcol = kind == 2 ? G.rhs_col + G.q + idx : (kind == 3 ? G.rhs_col + idx : -1);
    cplx v;
    if (r < 2 * l) {
      if (zcol >= 0) v = cmul(f, Zc[r + (int64_t)zcol * rsel]);
      else v = Psel[r + (int64_t)pcol * rsel];
      v = cmk(-v.x, -v.y);
      if (kind == 0 && C == r) v.x -= 1.0;
    } else if (r < 2 * l + rB) {
      const int ii = r - 2 * l;
      const int hcol = kind == 0 ? idx : (kind == 1 ? l + idx : (kind == 2 ? l + rB + G.q + idx : l + rB + idx));
      v = cmul(f, G.hc[ii + (int64_t)hcol * rB]);
      v = cmk(-v.x, -v.y);
      if (kind == 1 && idx == ii) v.x += 1.0;
    } else {
      const int tw = r - 2 * l - rB;
      const cplx* w = G.wd + (int64_t)tw * (M2 + rC) + M2;
      const cplx* X = zcol >= 0 ? EZ + (int64_t)zcol * S12 : EP + (int64_t)pcol * S12;
      cplx ph = wood_phi(DD, G, tw, X);
      cplx wz = cmk(0, 0);
      if (zcol >= 0)
        for (int c = 0; c < rC; ++c) wz = cfma(w[c], Zc[2 * l + c + (int64_t)zcol * rsel], wz);
      else
        for (int c = 0; c < rC; ++c) wz = cfma(w[c], Psel[2 * l + c + (int64_t)pcol * rsel], wz);
      v = cmul(f, csub(wz, ph));
      if (kind == 2) {
        cplx acc = cmk(0, 0);
        for (int sidx = D.S; sidx < 4 * D.S; ++sidx) {
          cplx p = wood_psi_tab(G, D.S, tw, sidx);
          if (p.x == 0.0 && p.y == 0.0) continue;
          acc = cfma(p, sample_point_pw(DD, G, idx, sidx, y0), acc);
        }
        v = cadd(v, acc);
      }
    }
    if (kind == 3) Rpool[G.r_off + (int64_t)idx * n + r] = v;
    else Spool[G.s_off + (int64_t)C * n + r] = v;
  }
}

// Sum_j A[j ld] x[j] for an FP64 column-strided A and a vector x in shared memory: in FP64,
// or (DF) in double-float on the FP32 pipes, A split on load and x already held as pairs,
// renormalised every 8 terms.  Eight loads of A are issued together ahead of their
// multiply-adds (each thread runs a long dot product alone; one load at a time would wait
// out the L2 latency at every term).
template <bool DF>
__device__ __forceinline__ cplx red_dot(const cplx* A, int64_t ld, const cplx* x, int n) {
  if constexpr (DF) {
    const dfc* xd = reinterpret_cast<const dfc*>(x);
    dfc acc{0.f, 0.f, 0.f, 0.f};
    int j = 0;
    for (; j + 8 <= n; j += 8) {
      cplx a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = A[(int64_t)(j + q) * ld];
#pragma unroll
      for (int q = 0; q < 8; ++q) dfc_mac_tile(to_dfc_bits(a[q]), xd[j + q], acc);
      dfc_norm(acc);
    }
    for (; j < n; ++j) dfc_mac_tile(to_dfc_bits(A[(int64_t)j * ld]), xd[j], acc);
    dfc_norm(acc);
    return from_dfc_bits(acc);
  } else {
    cplx acc = cmk(0, 0);
    int j = 0;
    for (; j + 8 <= n; j += 8) {
      cplx a[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) a[q] = A[(int64_t)(j + q) * ld];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc = cfma(a[q], x[j + q], acc);
    }
    for (; j < n; ++j) acc = cfma(A[(int64_t)j * ld], x[j], acc);
    return acc;
  }
}

// Entry i of a shared vector read by red_dot: FP64, or (DF) its double-float pair in place.
template <bool DF>
__device__ __forceinline__ void red_store(cplx* x, int i, cplx v) {
  if constexpr (DF) reinterpret_cast<dfc*>(x)[i] = to_dfc_bits(v);
  else x[i] = v;
}

// Bragg amplitudes from the reduced solution: gamma, xi = Q^{-1} U gamma, samples, DFT.
// The image columns of the neighbour unknowns enter as w = [alpha^{-1} u_1 + alpha u_2; u_B]
// (both images' columns of Z and of the E rows are the same skeleton columns).
template <bool DF>
__global__ void k_red_bragg(RedDims D, Dims DD, const GroupJob* groups, const AngleJob* angles, const cplx* Zc,
                            const cplx* Psel, const cplx* EZ, const cplx* EP, const cplx* Rpool, double y0,
                            cplx* cout, cplx* dout, double* flux) {
  extern __shared__ cplx sh[];
  const AngleJob A = angles[blockIdx.x];
  const GroupJob G = groups[A.group];
  const int l = D.l, rB = D.rB, rC = D.rC, rsel = D.rsel, S = D.S, S4 = 4 * D.S, S12 = 12 * D.S, M2 = 2 * D.M;
  const int n = G.nsys, nz = l + rB;
  cplx* w = sh;
  cplx* gam = sh + nz;
  cplx* xi = gam + rC;
  cplx* samp = xi + M2;
  const cplx* u = Rpool + G.r_off + (int64_t)A.col * n;
  const cplx ia = cdiv(cmk(1, 0), G.alpha);
  for (int j = threadIdx.x; j < nz; j += blockDim.x)
    red_store<DF>(w, j, j < l ? cadd(cmul(ia, u[j]), cmul(G.alpha, u[l + j])) : u[2 * l + (j - l)]);
  __syncthreads();
  for (int c = threadIdx.x; c < rC; c += blockDim.x) {
    const int row = 2 * l + c;
    cplx acc = red_dot<DF>(Zc + row, rsel, w, nz);
    for (int t = 0; t < G.nw; ++t) acc = cfma(Psel[row + (int64_t)(G.rhs_col + G.q + t) * rsel], u[2 * l + rB + t], acc);
    red_store<DF>(gam, c, csub(acc, Psel[row + (int64_t)(G.rhs_col + A.col) * rsel]));
  }
  __syncthreads();
  for (int mm = threadIdx.x; mm < M2; mm += blockDim.x) red_store<DF>(xi, mm, red_dot<DF>(G.qu + mm, M2, gam, rC));
  __syncthreads();
  for (int r = threadIdx.x; r < 2 * S; r += blockDim.x) {
    cplx acc = cmk(0, 0);
    cplx aj = ia;
    for (int jj = 0; jj < 3; ++jj) {
      const int row = S4 * jj + r;
      cplx part = csub(EP[row + (int64_t)(G.rhs_col + A.col) * S12], red_dot<DF>(EZ + row, S12, w, nz));
      for (int t = 0; t < G.nw; ++t)
        part = csub(part, cmul(EP[row + (int64_t)(G.rhs_col + G.q + t) * S12], u[2 * l + rB + t]));
      acc = cfma(aj, part, acc);
      aj = cmul(aj, G.alpha);
    }
    // the wall samples (SL + alpha SR) xi
    acc = cadd(acc, red_dot<DF>(G.sl + r, S4, xi, M2));
    acc = cfma(G.alpha, red_dot<DF>(G.sr + r, S4, xi, M2), acc);
    for (int t = 0; t < G.nw; ++t) acc = cfma(sample_point_pw(DD, G, t, r, y0), u[2 * l + rB + t], acc);
    samp[r] = acc;
  }
  __syncthreads();
  __shared__ double fl[32];
  const int no = A.n_max - A.n_min + 1;
  double fsum = 0.0;
  for (int o = threadIdx.x; o < no; o += blockDim.x) {
    const int nn = A.n_min + o;
    const double kap = A.kappa + 2.0 * HBS_PI * nn / D.d;
    cplx cn = cmk(0, 0), dn = cmk(0, 0);
    for (int si = 0; si < S; ++si) {
      const double xs = -0.5 * D.d + (si + 0.5) * D.d / S;
      double sn, cs;
      sincos(-kap * xs, &sn, &cs);
      cplx ev = cmk(cs / S, sn / S);
      cn = cfma(ev, samp[si], cn);
      dn = cfma(ev, samp[S + si], dn);
    }
    cout[A.out_off + o] = cn;
    dout[A.out_off + o] = dn;
    const double kn2 = D.omega * D.omega - kap * kap;
    const double kn = kn2 > 0 ? sqrt(kn2) : 0.0;
    cplx dd = dn;
    if (nn == 0) {
      double sn, cs;
      sincos(A.k0 * y0, &sn, &cs);
      dd = cadd(dd, cmk(cs, sn));
    }
    fsum += (kn / A.k0) * (cabs2(cn) + cabs2(dd));
  }
  for (int o = 16; o > 0; o >>= 1) fsum += __shfl_xor_sync(0xffffffffu, fsum, o);
  if ((threadIdx.x & 31) == 0) fl[threadIdx.x >> 5] = fsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += fl[w];
    flux[blockIdx.x] = fabs(t - 1.0);
  }
}

static AngleJob make_angle_job(double omega, double d, double th, int group, int col, int64_t* oo) {
  const double kap = omega * std::cos(th);
  AngleJob aj;
  aj.group = group;
  aj.col = col;
  aj.kappa = kap;
  aj.k0 = omega * std::fabs(std::sin(th));
  aj.n_min = (int)std::ceil((-omega - kap) * d / (2 * M_PI));
  aj.n_max = (int)std::floor((omega - kap) * d / (2 * M_PI));
  aj.out_off = *oo;
  *oo += aj.n_max - aj.n_min + 1;
  return aj;
}

// One batch of Bloch-phase groups on the precomputed, compressed path.
static void reduced_batch(Handle& h, std::vector<GroupJob>& gjobs, std::vector<std::vector<int64_t>*>& gmembers,
                          const double* theta, const cplx* Psel, int64_t cols, Result& out, cudaStream_t s) {
  const int l = h.nb_rank, M = h.M, S = h.S, rB = h.rB, rC = h.rC, rE = h.rE, rsel = h.rsel;
  const int M2 = 2 * M, S12 = 12 * S;
  const int ng = (int)gjobs.size();
  prof::PhaseSeq ph(s);
  ph.next("solve:schur");
  // E rows of the projections, expanded: EP = P_E Psel[E rows]
  DevBuf<cplx> EP((size_t)S12 * cols);
  {
    std::vector<GemmJob> gj(1);
    gj[0] = {h.PE.get(), Psel + 2 * l + rC, EP.get(), S12, (int)cols, rE, S12, rsel, S12, cmk(1, 0), cmk(0, 0), 0, 0, 0};
    run_gemms(gj, s);
  }
  // per-group work arrays
  int64_t nvt = 0, nqu = 0, nhm = 0, nhc = 0, nwd = 0, nps = 0, so = 0, ro = 0;
  for (auto& G : gjobs) {
    G.nsys = 2 * l + rB + G.nw;
    nps += (int64_t)G.nw * 3 * S;
    nvt += (int64_t)rB * M2;
    nqu += (int64_t)M2 * rC;
    nhm += (int64_t)rB * rC;
    nhc += (int64_t)rB * (l + rB + G.q + G.nw);
    nwd += (int64_t)G.nw * (M2 + rC);
    G.s_off = so; so += (int64_t)G.nsys * G.nsys;
    G.r_off = ro; ro += (int64_t)G.nsys * G.q;
  }
  DevBuf<cplx> vt(std::max<int64_t>(nvt, 1)), qu(std::max<int64_t>(nqu, 1)), hm(std::max<int64_t>(nhm, 1)),
      hc(std::max<int64_t>(nhc, 1)), wd(std::max<int64_t>(nwd, 1)), Sp(std::max<int64_t>(so, 1)),
      Rp(std::max<int64_t>(ro, 1)), qcoef((size_t)ng * 5 * M), wpsi(std::max<int64_t>(nps, 1));
  {
    int64_t a = 0, b = 0, c = 0, d2 = 0, e = 0, f = 0;
    for (size_t gg = 0; gg < gjobs.size(); ++gg) {
      GroupJob& G = gjobs[gg];
      G.qcoef = qcoef.get() + 5 * (int64_t)M * gg;
      G.wpsi = wpsi.get() + f; f += (int64_t)G.nw * 3 * S;
      const ContourData& cd = h.contours[G.contour];
      G.ul = cd.UL.get(); G.ur = cd.UR.get(); G.vl = cd.VL.get(); G.vr = cd.VR.get();
      G.vt = vt.get() + a; a += (int64_t)rB * M2;
      G.qu = qu.get() + b; b += (int64_t)M2 * rC;
      G.hm = hm.get() + c; c += (int64_t)rB * rC;
      G.hc = hc.get() + d2; d2 += (int64_t)rB * (l + rB + G.q + G.nw);
      G.wd = wd.get() + e; e += (int64_t)G.nw * (M2 + rC);
    }
  }
  DevBuf<GroupJob> dg;
  dg.upload(gjobs, s);
  RedDims R{l, M, S, rB, rC, rsel, h.d, h.omega};
  Dims DD{l, M, S, 0, h.d, h.omega, 0};
  {
    prof::KScope _ks("k_red_tables", s);
    k_red_tables<<<dim3((M + 12 * S + 255) / 256, ng), 256, 0, s>>>(R, DD, dg.get());
  }
  HBS_LAUNCH_CHECK("k_red_tables");
  {
    prof::KScope _ks("k_red_prep", s);
    k_red_prep<<<dim3(64, ng), 256, 0, s>>>(R, dg.get());
  }
  HBS_LAUNCH_CHECK("k_red_prep");
  {
    std::vector<GemmJob> gj;
    for (auto& G : gjobs)
      gj.push_back({G.vt, G.qu, G.hm, rB, rC, M2, rB, M2, rB, cmk(1, 0), cmk(0, 0), 0, 0, 0});
    run_gemms(gj, s);
    gj.clear();
    for (auto& G : gjobs) {
      gj.push_back({G.hm, h.Zc.get() + 2 * l, G.hc, rB, l + rB, rC, rB, rsel, rB, cmk(1, 0), cmk(0, 0), 0, 0, 0});
      gj.push_back({G.hm, Psel + 2 * l + (int64_t)G.rhs_col * rsel, G.hc + (int64_t)(l + rB) * rB, rB, G.q + G.nw, rC,
                    rB, rsel, rB, cmk(1, 0), cmk(0, 0), 0, 0, 0});
    }
    run_gemms(gj, s);
  }
  {
    prof::KScope _ks("k_red_wood", s);
    k_red_wood<<<ng, 256, 0, s>>>(R, dg.get(), DD);
  }
  {
    prof::KScope _ks("k_red_assemble", s);
    k_red_assemble<<<dim3(64, ng), 256, 0, s>>>(R, DD, dg.get(), h.Zc.get(), Psel, h.EZ.get(), EP.get(), h.y0,
                                                 Sp.get(), Rp.get());
  }
  HBS_LAUNCH_CHECK("k_red_assemble");
  DevBuf<int> ill(ng);
  {
    double sfl = 0.0;
    for (auto& G : gjobs) {
      const double n = G.nsys;
      sfl += 8.0 / 3.0 * n * n * n + 8.0 * n * n * G.q;
    }
    prof::KScope _ks("k_schur_solve", s, sfl, 0.0);
    schur_solve(DD, gjobs, dg.get(), Sp.get(), Rp.get(), ill.get(), s);
  }
  HBS_LAUNCH_CHECK("k_schur_solve");
  ph.next("solve:bragg");
  std::vector<AngleJob> ajobs;
  int64_t oo = 0;
  for (int gg = 0; gg < ng; ++gg) {
    const auto& mem = *gmembers[gg];
    for (int a = 0; a < gjobs[gg].q; ++a) ajobs.push_back(make_angle_job(h.omega, h.d, theta[mem[a]], gg, a, &oo));
  }
  DevBuf<AngleJob> da;
  da.upload(ajobs, s);
  DevBuf<cplx> cbuf(std::max<int64_t>(oo, 1)), dbuf(std::max<int64_t>(oo, 1));
  DevBuf<double> fbuf(ajobs.size());
  {
    prof::KScope _ks("k_red_bragg", s);
    const size_t shm = (size_t)(l + rB + rC + M2 + 2 * S) * sizeof(cplx);
    // double-float products on double-float handles (the FP64 pipe's rate bounds this kernel)
    const bool df = gemm_double_float();
    const void* fn = df ? (const void*)k_red_bragg<true> : (const void*)k_red_bragg<false>;
    HBS_CUDA(raise_smem_limit(fn, shm));
    if (df)
      k_red_bragg<true><<<(unsigned)ajobs.size(), 128, shm, s>>>(R, DD, dg.get(), da.get(), h.Zc.get(), Psel,
                                                                 h.EZ.get(), EP.get(), Rp.get(), h.y0, cbuf.get(),
                                                                 dbuf.get(), fbuf.get());
    else
      k_red_bragg<false><<<(unsigned)ajobs.size(), 128, shm, s>>>(R, DD, dg.get(), da.get(), h.Zc.get(), Psel,
                                                                  h.EZ.get(), EP.get(), Rp.get(), h.y0, cbuf.get(),
                                                                  dbuf.get(), fbuf.get());
  }
  HBS_LAUNCH_CHECK("k_red_bragg");
  auto hcv = cbuf.download(s), hdv = dbuf.download(s);
  auto hf = fbuf.download(s);
  auto hill = ill.download(s);
  for (int v : hill)
    if (v) out.illcond = true;
  size_t ai = 0;
  for (int gg = 0; gg < ng; ++gg) {
    const auto& mem = *gmembers[gg];
    for (int a = 0; a < gjobs[gg].q; ++a, ++ai) {
      const AngleJob& aj = ajobs[ai];
      AngleResult& r = out.angles[mem[a]];
      r.n_min = aj.n_min;
      r.n_max = aj.n_max;
      const int no = aj.n_max - aj.n_min + 1;
      r.c.resize(no);
      r.d.resize(no);
      for (int o = 0; o < no; ++o) {
        r.c[o] = zc(hcv[aj.out_off + o].x, hcv[aj.out_off + o].y);
        r.d[o] = zc(hdv[aj.out_off + o].x, hdv[aj.out_off + o].y);
      }
      r.flux_err = hf[ai];
      r.n_wood = gjobs[gg].nw;
      r.t0 = h.contours[gjobs[gg].contour].t0;
    }
  }
}

// k_n = sqrt(w^2 - kappa_n^2) (non-negative real or positive imaginary).  An order within
// rounding of a Rayleigh-Wood anomaly (|w^2 - kappa_n^2| <= 1e-12 w^2; an angle given as the
// anomaly in FP64 lands there) is taken at the anomaly, k_n = 0: the amplitudes have a
// square-root singularity in the angle there, so the few-ulp differences between ways of
// forming kappa_n would otherwise show up at the 1e-8 level.
static zc kn_of(double omega, double kap) {
  double v = omega * omega - kap * kap;
  if (std::fabs(v) <= 1e-12 * omega * omega) return zc(0.0, 0.0);
  return v >= 0 ? zc(std::sqrt(v), 0.0) : zc(0.0, std::sqrt(-v));
}

// Full wall rows C_L^c, C_R^c and Bragg sampling rows E, used only by the plain path.
static void ensure_full_rows(Handle& h, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(h.lazy_mu);
  const int64_t N = h.N;
  const int M = h.M, S = h.S;
  const DevGeom g = Handle_geom(h);
  if (!h.Esamp.get()) {
    h.Esamp.alloc((size_t)12 * S * N);
    for (int jj = 0; jj < 3; ++jj) {
      prof::KScope _ks("k_fill_samples", s);
      k_fill_samples<<<grid_1d((int64_t)4 * S * N), 256, 0, s>>>(g, S, h.d, h.y0, (jj - 1) * h.d,
                                                                   h.Esamp.get() + 4 * S * jj, 12 * S);
    }
    HBS_LAUNCH_CHECK("k_fill_samples");
  }
  for (auto& cd : h.contours) {
    if (cd.CL.get()) continue;
    cd.CL.alloc((size_t)2 * M * N);
    cd.CR.alloc((size_t)2 * M * N);
    prof::KScope _ks("k_fill_c", s);
    k_fill_c<<<grid_1d(N * (int64_t)M), 256, 0, s>>>(g, cd.dk.get(), M, h.d, -0.5 * h.d, cd.CL.get(), 2 * M);
    k_fill_c<<<grid_1d(N * (int64_t)M), 256, 0, s>>>(g, cd.dk.get(), M, -h.d, 0.5 * h.d, cd.CR.get(), 2 * M);
  }
  HBS_LAUNCH_CHECK("k_fill_c");
  HBS_CUDA(cudaStreamSynchronize(s));
}

void solve_angles(Handle& h, const double* theta, int64_t n_theta, bool plain, Result& out, cudaStream_t s) {
  if (plain) ensure_full_rows(h, s);
  const double omega = h.omega, d = h.d;
  const int l = h.nb_rank, M = h.M, S = h.S;
  const int zr = 2 * l + 4 * M + 12 * S;
  const DevGeom g = Handle_geom(h);
  out.angles.assign(n_theta, AngleResult());
  out.illcond = false;
  if (n_theta == 0) return;
  for (int64_t i = 0; i < n_theta; ++i)
    if (!(theta[i] > -M_PI && theta[i] < 0.0)) throw Error(HBS_ERR_INVALID_ARG, "incident angle outside (-pi, 0)");

  // ---- group angles by Bloch phase (Remark 3.1)
  std::vector<int64_t> order(n_theta);
  std::vector<double> key(n_theta);
  for (int64_t i = 0; i < n_theta; ++i) {
    double ph = std::fmod(omega * d * std::cos(theta[i]), 2.0 * M_PI);
    if (ph < 0) ph += 2.0 * M_PI;
    key[i] = ph;
    order[i] = i;
  }
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  std::vector<std::vector<int64_t>> groups;
  for (int64_t t = 0; t < n_theta; ++t) {
    int64_t i = order[t];
    if (!groups.empty()) {
      double k0 = key[groups.back()[0]];
      double dk = std::fabs(key[i] - k0);
      dk = std::min(dk, 2.0 * M_PI - dk);
      if (dk < 1e-9) { groups.back().push_back(i); continue; }
    }
    groups.push_back({i});
  }
  // wrap-around merge (phase near 0 and near 2 pi)
  if (groups.size() > 1) {
    double a = key[groups.front()[0]], b = key[groups.back()[0]];
    if (std::fabs(a + 2.0 * M_PI - b) < 1e-9) {
      for (auto i : groups.back()) groups.front().push_back(i);
      groups.pop_back();
    }
  }

  // ---- process groups in batches
  const int nc = (int)h.contours.size();
  // Columns per batch of groups: the precomputed path keeps only rsel x cols
  // projections per batch, so all groups of a typical call share one Schur launch.
  const int64_t max_cols = plain ? 1024 : 8192;
  size_t gi = 0;
  while (gi < groups.size()) {
    std::vector<GroupJob> gjobs;
    std::vector<AngleJob> ajobs;
    std::vector<RhsCol> rcols;
    std::vector<std::vector<int64_t>*> gmembers;
    int64_t cols = 0;
    while (gi < groups.size()) {
      auto& mem = groups[gi];
      const int q = (int)mem.size();
      const double th0 = theta[mem[0]];
      const double kap_i = omega * std::cos(th0);
      // poles +-k_n of the integrand: choose the contour that stays farther from all of
      // them (distance in the trapezoid variable t), since the trapezoid rule loses
      // accuracy like exp(-2 pi dist / h) as a pole approaches the contour.  Distances
      // beyond 3 count as 3 (both contours are then exact to rounding); on a tie the
      // standard contour is kept.
      std::vector<std::pair<int, zc>> modes;
      const int nlo = (int)std::floor((-omega - kap_i) * d / (2 * M_PI)) - 4;
      const int nhi = (int)std::ceil((omega - kap_i) * d / (2 * M_PI)) + 4;
      const double t1 = nc > 1 ? h.contours[1].t0 : 0.0;
      double dist[2] = {3.0, 3.0};
      for (int n = nlo; n <= nhi; ++n) {
        zc kn = kn_of(omega, kap_i + 2 * M_PI * n / d);
        modes.push_back({n, kn});
        // only poles near a crossing point (0 or t1) can come close to either contour
        if (std::fabs(kn.real()) > std::max(t1, 0.0) + 6.0) continue;
        for (int cc = 0; cc < nc; ++cc)
          dist[cc] = std::min(dist[cc], std::min(contour_distance(h, cc, kn), contour_distance(h, cc, -kn)));
      }
      const int c = (nc > 1 && dist[1] > dist[0]) ? 1 : 0;
      GroupJob G{};
      std::vector<std::pair<double, zc>> wood;
      if (c == 1) {
        const double height = h.cc * std::tanh(t1 / h.cw);
        for (auto& md : modes) {
          zc kn = md.second;
          bool flip = (kn.imag() == 0.0) ? (kn.real() >= 0.0 && kn.real() < t1) : (kn.real() == 0.0 && kn.imag() < height);
          if (flip) wood.push_back({kap_i + 2 * M_PI * md.first / d, kn});
        }
      }
      if (wood.size() > 4) throw Error(HBS_ERR_INTERNAL, "more than four Wood's modes flipped");
      const int nw = (int)wood.size();
      const int need = q + nw + (plain ? 2 * l + 2 * M : 0);
      if (!gjobs.empty() && cols + need > max_cols) break;
      G.alpha = to_c(std::exp(zc(0.0, omega * d * std::cos(th0))));
      G.q = q;
      G.nw = nw;
      G.rhs_col = (int)cols;
      G.contour = c;
      G.zp = h.contours[c].Zd.get();
      G.sl = h.contours[c].SL.get();
      G.sr = h.contours[c].SR.get();
      G.ck = h.contours[c].dk.get();
      for (int t = 0; t < nw; ++t) { G.wkap[t] = wood[t].first; G.wkn[t] = to_c(wood[t].second); }
      for (int a = 0; a < q; ++a) {
        const double th = theta[mem[a]];
        rcols.push_back({omega * std::cos(th), cmk(omega * std::sin(th), 0.0), -1.0});
      }
      for (int t = 0; t < nw; ++t) rcols.push_back({wood[t].first, to_c(wood[t].second), 1.0});
      cols += q + nw;
      if (plain) cols += 2 * l + 2 * M;
      gjobs.push_back(G);
      gmembers.push_back(&mem);
      ++gi;
    }
    const int ng = (int)gjobs.size();
    const int64_t N = h.N;
    prof::PhaseSeq ph(s);
    if (!plain) {
      // Precomputed path: Rsel A^{-1} [b | PW] = V [b | PW] with V^T = A^{-T} Rsel^T formed at
      // build.  Incident-field columns and propagating Wood's plane waves come from V on
      // plane waves in K equispaced directions by trigonometric interpolation in the
      // direction angle: V e^{i k.x} = e^{i k.c} sum_k P_k D_K(psi - phi_k), D_K the
      // interpolation kernel of K equispaced points.  Evanescent Wood's columns (complex
      // k_n) are formed directly.  The reduced Schur systems work on these projections.
      ph.next("solve:projections");
      int64_t pos = 0;
      for (auto& G : gjobs) { G.rhs_col = (int)pos; pos += G.q + G.nw; }
      const int K = h.Kdir;
      DevBuf<cplx> Psel((size_t)h.rsel * cols);
      // per column: the direction angle and phase of its plane wave (propagating), or a zero
      // phase (evanescent: formed directly below); the weights are formed on the device
      std::vector<double> hpsi((size_t)cols, 0.0);
      std::vector<cplx> hphase((size_t)cols, cmk(0, 0));
      std::vector<RhsCol> evan;
      std::vector<int64_t> evan_col;
      size_t rc = 0;
      for (int gg = 0; gg < ng; ++gg) {
        const GroupJob& G = gjobs[gg];
        for (int a2 = 0; a2 < G.q + G.nw; ++a2, ++rc) {
          const RhsCol& r = rcols[rc];
          const int64_t col = G.rhs_col + a2;
          if (r.ky.y == 0.0) {
            hpsi[col] = std::atan2(r.ky.x, r.kap);
            const zc phase = r.sign * std::exp(zc(0.0, r.kap * h.dir_cx + r.ky.x * h.dir_cy));
            hphase[col] = to_c(phase);
          } else {
            evan.push_back(r);
            evan_col.push_back(col);
          }
        }
      }
      DevBuf<double> dpsi;
      DevBuf<cplx> dphase, dint((size_t)K * cols);
      dpsi.upload(hpsi, s);
      dphase.upload(hphase, s);
      {
        prof::KScope _ks("k_interp_dirs", s);
        k_interp_dirs<<<grid_1d((int64_t)K * cols), 256, 0, s>>>(dpsi.get(), dphase.get(), cols, K, dint.get());
      }
      HBS_LAUNCH_CHECK("k_interp_dirs");
      std::vector<GemmJob> gj(1);
      gj[0] = {h.Pdir.get(), dint.get(), Psel.get(), h.rsel, (int)cols, K, h.rsel, K, h.rsel, cmk(1, 0), cmk(0, 0), 0,
               0, 0, 0};
      run_gemms(gj, s);
      if (!evan.empty()) {
        const int ne = (int)evan.size();
        DevBuf<cplx> RHSe((size_t)N * ne), Pe((size_t)h.rsel * ne);
        DevBuf<RhsCol> dr;
        dr.upload(evan, s);
        {
          prof::KScope _ks("k_fill_rhs", s);
          k_fill_rhs<<<grid_1d(N * ne), 256, 0, s>>>(g, dr.get(), ne, RHSe.get());
        }
        HBS_LAUNCH_CHECK("k_fill_rhs");
        gj[0] = {h.VT.get(), RHSe.get(), Pe.get(), h.rsel, ne, (int)N, (int)N, (int)N, h.rsel, cmk(1, 0), cmk(0, 0), 0,
                 0, 0, 1};
        run_gemms(gj, s);
        for (int e = 0; e < ne; ++e)
          HBS_CUDA(cudaMemcpyAsync(Psel.get() + evan_col[e] * h.rsel, Pe.get() + (int64_t)e * h.rsel,
                                   sizeof(cplx) * h.rsel, cudaMemcpyDeviceToDevice, s));
        HBS_CUDA(cudaStreamSynchronize(s));
      }
      ph.close();
      reduced_batch(h, gjobs, gmembers, theta, Psel.get(), cols, out, s);
      continue;
    }
    ph.next("solve:rhs_apply");
    // ---- right-hand sides, applies
    DevBuf<cplx> RHS((size_t)N * cols), X((size_t)N * cols);
    {
      // b and PW columns are packed per group at rhs_col; in the plain path the
      // L and B(alpha) columns follow each group's q + nw columns.
      int64_t pos = 0;
      size_t rc = 0;
      for (int gg = 0; gg < ng; ++gg) {
        GroupJob& G = gjobs[gg];
        G.rhs_col = (int)pos;
        DevBuf<RhsCol> dr;
        dr.upload(std::vector<RhsCol>(rcols.begin() + rc, rcols.begin() + rc + G.q + G.nw), s);
        rc += G.q + G.nw;
        {
          prof::KScope _ks("k_fill_rhs", s);
          k_fill_rhs<<<grid_1d(N * (G.q + G.nw)), 256, 0, s>>>(g, dr.get(), G.q + G.nw, RHS.get() + pos * N);
        }
        HBS_LAUNCH_CHECK("k_fill_rhs");
        HBS_CUDA(cudaStreamSynchronize(s));
        pos += G.q + G.nw;
        if (plain) {
          // L = [alpha^{-1} P | alpha P], B(alpha) = B_L + alpha B_R
          const cplx ia = cdiv(cmk(1, 0), G.alpha);
          if (l > 0) {
            {
              prof::KScope _ks("k_scaled_copy", s);
              k_scaled_copy<<<grid_1d(N * l), 256, 0, s>>>(h.Pnb.get(), N * (int64_t)l, ia, RHS.get() + pos * N);
            }
            {
              prof::KScope _ks("k_scaled_copy", s);
              k_scaled_copy<<<grid_1d(N * l), 256, 0, s>>>(h.Pnb.get(), N * (int64_t)l, G.alpha, RHS.get() + (pos + l) * N);
            }
          }
          const ContourData& cd = h.contours[G.contour];
          {
            prof::KScope _ks("k_fill_b", s);
            k_fill_b<<<grid_1d(N * (int64_t)M), 256, 0, s>>>(g, cd.dk.get(), cd.dwk.get(), M, d, RHS.get(), N, pos + 2 * l,
                                                              0, 1, G.alpha);
          }
          HBS_LAUNCH_CHECK("plain fills");
          pos += 2 * l + 2 * M;
        }
      }
    }

    h.apply_inverse(RHS.get(), X.get(), cols, s);
    RHS.release();
    // ---- Proj = Rows X
    ph.next("solve:projections");
    DevBuf<cplx> Proj((size_t)zr * cols);
    {
      std::vector<GemmJob> gj;
      for (int gg = 0; gg < ng; ++gg) {
        const GroupJob& G = gjobs[gg];
        const ContourData& cd = h.contours[G.contour];
        const int gcols = G.q + G.nw + (plain ? 2 * l + 2 * M : 0);
        struct Blk { const cplx* A; int rows; int lda; int row0; };
        Blk rows[5] = {{h.Rm.get(), l, l, 0}, {h.Rp.get(), l, l, l}, {cd.CL.get(), 2 * M, 2 * M, 2 * l},
                       {cd.CR.get(), 2 * M, 2 * M, 2 * l + 2 * M}, {h.Esamp.get(), 12 * S, 12 * S, 2 * l + 4 * M}};
        for (auto& rb : rows) {
          if (rb.rows == 0) continue;
          gj.push_back({rb.A, X.get() + (int64_t)G.rhs_col * N, Proj.get() + (int64_t)G.rhs_col * zr + rb.row0, rb.rows,
                        gcols, (int)N, rb.lda, (int)N, zr, cmk(1, 0), cmk(0, 0), 0, 0, 0});
        }
      }
      run_gemms(gj, s);
    }
    X.release();
    // plain path: point zl / zb at the per-group products
    for (int gg = 0; gg < ng; ++gg) {
      GroupJob& G = gjobs[gg];
      if (plain) {
        G.zl = Proj.get() + (int64_t)(G.rhs_col + G.q + G.nw) * zr;
        G.zb = Proj.get() + (int64_t)(G.rhs_col + G.q + G.nw + 2 * l) * zr;
      }
    }
    // ---- Schur systems
    ph.next("solve:schur");
    int64_t so = 0, ro = 0;
    for (auto& G : gjobs) {
      const int nS = 2 * l + 2 * M + G.nw;
      G.nsys = nS;
      G.s_off = so; so += (int64_t)nS * nS;
      G.r_off = ro; ro += (int64_t)nS * G.q;
    }
    DevBuf<cplx> Sp(so), Rp(ro);
    DevBuf<GroupJob> dg;
    dg.upload(gjobs, s);
    Dims D{l, M, S, zr, d, omega, zr};
    {
      prof::KScope _ks("k_assemble", s);
      k_assemble<<<dim3(64, ng), 256, 0, s>>>(D, dg.get(), Proj.get(), h.y0, Sp.get(), Rp.get());
    }
    HBS_LAUNCH_CHECK("k_assemble");
    DevBuf<int> ill(ng);
    double sfl = 0.0;
    for (auto& G : gjobs) {
      const double n = 2.0 * l + 2.0 * M + G.nw;
      sfl += 8.0 / 3.0 * n * n * n + 8.0 * n * n * G.q;
    }
    {
      prof::KScope _ks("k_schur_solve", s, sfl, 0.0);
      schur_solve(D, gjobs, dg.get(), Sp.get(), Rp.get(), ill.get(), s);
    }
    HBS_LAUNCH_CHECK("k_schur_solve");
    // ---- Bragg amplitudes
    ph.next("solve:bragg");
    int64_t oo = 0;
    for (int gg = 0; gg < ng; ++gg) {
      const auto& mem = *gmembers[gg];
      for (int a = 0; a < gjobs[gg].q; ++a) {
        const double th = theta[mem[a]];
        const double kap = omega * std::cos(th);
        AngleJob aj;
        aj.group = gg;
        aj.col = a;
        aj.kappa = kap;
        aj.k0 = omega * std::fabs(std::sin(th));
        aj.n_min = (int)std::ceil((-omega - kap) * d / (2 * M_PI));
        aj.n_max = (int)std::floor((omega - kap) * d / (2 * M_PI));
        aj.out_off = oo;
        oo += aj.n_max - aj.n_min + 1;
        ajobs.push_back(aj);
      }
    }
    DevBuf<AngleJob> da;
    da.upload(ajobs, s);
    DevBuf<cplx> cbuf(std::max<int64_t>(oo, 1)), dbuf(std::max<int64_t>(oo, 1));
    DevBuf<double> fbuf(ajobs.size());
    {
      prof::KScope _ks("k_bragg", s);
      k_bragg<<<(unsigned)ajobs.size(), 128, 2 * S * sizeof(cplx), s>>>(D, dg.get(), da.get(), Proj.get(), Rp.get(), h.y0,
                                                                        cbuf.get(), dbuf.get(), fbuf.get());
    }
    HBS_LAUNCH_CHECK("k_bragg");
    auto hc = cbuf.download(s), hd = dbuf.download(s);
    auto hf = fbuf.download(s);
    auto hill = ill.download(s);
    for (int v : hill)
      if (v) out.illcond = true;
    size_t ai = 0;
    for (int gg = 0; gg < ng; ++gg) {
      const auto& mem = *gmembers[gg];
      for (int a = 0; a < gjobs[gg].q; ++a, ++ai) {
        const AngleJob& aj = ajobs[ai];
        AngleResult& r = out.angles[mem[a]];
        r.n_min = aj.n_min;
        r.n_max = aj.n_max;
        const int no = aj.n_max - aj.n_min + 1;
        r.c.resize(no);
        r.d.resize(no);
        for (int o = 0; o < no; ++o) {
          r.c[o] = zc(hc[aj.out_off + o].x, hc[aj.out_off + o].y);
          r.d[o] = zc(hd[aj.out_off + o].x, hd[aj.out_off + o].y);
        }
        r.flux_err = hf[ai];
        r.n_wood = gjobs[gg].nw;
        r.t0 = h.contours[gjobs[gg].contour].t0;
      }
    }
  }
}

}  // namespace hbs
