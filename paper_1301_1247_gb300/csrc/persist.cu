// hbs_save / hbs_load: a built solver written to and read back from a file, so that a
// serving process can keep factors of many geometries without rebuilding them.
//
// Format (native byte order; the file is for the machine that wrote it):
//   8-byte magic "HBSQP\0v1", then the sizes of the option struct and of the element
//   types as a compatibility check, then every field of the handle in a fixed order
//   (scalars raw, host arrays and device buffers as a 64-bit element count followed by
//   the elements).  The lazily formed dense rows of the plain path are not stored.
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>

#include "dense_kernels.cuh"
#include "handle.hpp"
#include "qp_kernels.cuh"

namespace hbs {

namespace {

constexpr char kMagic[8] = {'H', 'B', 'S', 'Q', 'P', '\0', 'v', '1'};

struct FileCloser {
  void operator()(FILE* f) const {
    if (f) std::fclose(f);
  }
};
using File = std::unique_ptr<FILE, FileCloser>;

struct Writer {
  FILE* f;
  cudaStream_t s;
  void bytes(const void* p, size_t n) {
    if (n && std::fwrite(p, 1, n, f) != n) throw Error(HBS_ERR_IO, "write failed");
  }
  template <typename T>
  void pod(T& v) {
    bytes(&v, sizeof(T));
  }
  template <typename T>
  void vec(std::vector<T>& v) {
    uint64_t n = v.size();
    pod(n);
    bytes(v.data(), n * sizeof(T));
  }
  template <typename T>
  void dev(DevBuf<T>& b) {
    uint64_t n = b.size();
    pod(n);
    if (n) {
      std::vector<T> h = b.download(s);
      bytes(h.data(), n * sizeof(T));
    }
  }
  template <typename T>
  void count(std::vector<T>& v) {
    uint64_t n = v.size();
    pod(n);
  }
};

struct Reader {
  FILE* f;
  cudaStream_t s;
  void bytes(void* p, size_t n) {
    if (n && std::fread(p, 1, n, f) != n) throw Error(HBS_ERR_IO, "file is truncated or unreadable");
  }
  uint64_t length(size_t elem) {
    uint64_t n = 0;
    bytes(&n, sizeof n);
    if (n > (uint64_t(1) << 40) / elem) throw Error(HBS_ERR_IO, "corrupt length in file");
    return n;
  }
  template <typename T>
  void pod(T& v) {
    bytes(&v, sizeof(T));
  }
  template <typename T>
  void vec(std::vector<T>& v) {
    v.resize(length(sizeof(T)));
    bytes(v.data(), v.size() * sizeof(T));
  }
  template <typename T>
  void dev(DevBuf<T>& b) {
    std::vector<T> h(length(sizeof(T)));
    bytes(h.data(), h.size() * sizeof(T));
    b.release();
    if (!h.empty()) {
      b.alloc(h.size());
      HBS_CUDA(cudaMemcpyAsync(b.get(), h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
      HBS_CUDA(cudaStreamSynchronize(s));  // h goes out of scope
    }
  }
  template <typename T>
  void count(std::vector<T>& v) {
    v.resize(length(1));
  }
};

// Every persistent field of the handle, in file order.
template <class Ar>
void visit(Ar& ar, Handle& h) {
  ar.pod(h.N);
  ar.pod(h.nodes); ar.pod(h.comps); ar.pod(h.index);
  ar.pod(h.d);
  ar.pod(h.omega);
  ar.pod(h.tol);
  ar.pod(h.opts);
  ar.pod(h.L);
  ar.dev(h.x); ar.dev(h.y); ar.dev(h.nx); ar.dev(h.ny); ar.dev(h.w);
  ar.vec(h.hx); ar.vec(h.hy); ar.vec(h.hnx); ar.vec(h.hny); ar.vec(h.hw);
  ar.count(h.levels);
  for (Level& lv : h.levels) {
    ar.pod(lv.l); ar.pod(lv.first); ar.pod(lv.count);
    ar.vec(lv.n); ar.vec(lv.k); ar.vec(lv.off); ar.pod(lv.ntot);
    ar.dev(lv.idx); ar.dev(lv.perm); ar.vec(lv.t_off); ar.dev(lv.T);
    ar.vec(lv.e_off); ar.vec(lv.f_off); ar.vec(lv.g_off); ar.vec(lv.dh_off);
    ar.dev(lv.E); ar.dev(lv.F); ar.dev(lv.G); ar.dev(lv.Dhat);
    ar.dev(lv.cx); ar.dev(lv.cy); ar.dev(lv.rad); ar.vec(lv.h_rad);
    ar.pod(lv.passthru);
  }
  ar.pod(h.nroot); ar.dev(h.Groot); ar.pod(h.max_rank);
  ar.pod(h.nb_rank); ar.pod(h.nb_R); ar.pod(h.nb_np);
  ar.dev(h.nb_skel); ar.dev(h.Pnb); ar.dev(h.Rm); ar.dev(h.Rp);
  ar.pod(h.S); ar.pod(h.y0);
  ar.pod(h.M); ar.pod(h.ch); ar.pod(h.cc); ar.pod(h.cw); ar.pod(h.cK);
  ar.count(h.contours);
  for (ContourData& c : h.contours) {
    ar.pod(c.t0); ar.vec(c.k); ar.vec(c.wk); ar.dev(c.dk); ar.dev(c.dwk); ar.pod(c.col_off);
    ar.dev(c.SL); ar.dev(c.SR); ar.pod(c.zr); ar.pod(c.zc);
    ar.dev(c.row_recipe); ar.dev(c.col_recipe);
    ar.dev(c.UL); ar.dev(c.UR); ar.dev(c.VL); ar.dev(c.VR);
  }
  ar.pod(h.wcols); ar.pod(h.rB); ar.pod(h.rC); ar.pod(h.rE); ar.pod(h.rsel);
  ar.dev(h.TY); ar.dev(h.TC); ar.dev(h.TE); ar.dev(h.Rsel); ar.dev(h.VT); ar.dev(h.Zc); ar.dev(h.PE); ar.dev(h.EZ);
  ar.dev(h.Pdir); ar.pod(h.Kdir); ar.pod(h.dir_cx); ar.pod(h.dir_cy);
  ar.pod(h.pid_residual); ar.pod(h.nb_residual);
  ar.pod(h.build_seconds); ar.pod(h.factor_bytes); ar.pod(h.apply_flops);
}

struct Header {
  char magic[8];
  uint32_t opts_bytes, cplx_bytes, int2_bytes, handle_fields;
};

Header make_header() {
  Header hd{};
  std::memcpy(hd.magic, kMagic, sizeof kMagic);
  hd.opts_bytes = (uint32_t)sizeof(hbs_options);
  hd.cplx_bytes = (uint32_t)sizeof(cplx);
  hd.int2_bytes = (uint32_t)sizeof(int2);
  hd.handle_fields = 3;  // layout revision of visit()
  return hd;
}

}  // namespace

void save_handle(Handle& h, const char* path, cudaStream_t s) {
  File f(std::fopen(path, "wb"));
  if (!f) throw Error(HBS_ERR_IO, std::string("cannot open ") + path + " for writing");
  Writer w{f.get(), s};
  Header hd = make_header();
  w.pod(hd);
  visit(w, h);
  if (std::fflush(f.get()) != 0) throw Error(HBS_ERR_IO, "write failed");
}

void load_handle(Handle& h, const char* path, cudaStream_t s) {
  File f(std::fopen(path, "rb"));
  if (!f) throw Error(HBS_ERR_IO, std::string("cannot open ") + path);
  Reader r{f.get(), s};
  Header hd{};
  r.pod(hd);
  const Header want = make_header();
  if (std::memcmp(&hd, &want, sizeof hd) != 0) throw Error(HBS_ERR_IO, "not a solver file of this library version");
  visit(r, h);
  int probe = 0;
  if (std::fread(&probe, 1, 1, f.get()) != 0) throw Error(HBS_ERR_IO, "trailing bytes after the solver data");
}

}  // namespace hbs
