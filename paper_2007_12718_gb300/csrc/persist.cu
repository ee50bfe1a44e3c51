// Reuse and persistence of built data.
//
// * The compression (Sec. 3.2) depends on the kernel, the lattice and the
//   boxes, not on the potential b: the per-level skeletons, the interpolation
//   matrices U, the sibling blocks and their low-rank factors are the same for
//   every b on a grid with the same kappa, h, tree, tolerance, quadrature order
//   and ring (the paper notes that this compression can be computed once and
//   stored).  With ls_opts.reuse_compression = 1, ls_build keeps a device copy
//   of them per key in a process-wide cache and a later build with the same key
//   copies them into its handle instead of compressing: only the leaf build and
//   the merges (which carry b) run.
// * ls_save / ls_load write a built handle to a file and restore it: the inputs
//   and every factor, so that a later process applies and solves without
//   compressing or merging.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "handle.h"

namespace ls {
namespace {

size_t elem_bytes(const ls_handle* H) { return H->prec == LS_FP64 ? sizeof(z64) : sizeof(c32); }

// ------------------------------------------------------------- the cache
struct CacheKey {
  int device, nx, ny, s, L, ring, order_precond, precision, top_uncompressed, id_method, woodbury;
  double kappa, h, tol;
  bool operator==(const CacheKey& o) const {
    return device == o.device && nx == o.nx && ny == o.ny && s == o.s && L == o.L && ring == o.ring &&
           order_precond == o.order_precond && precision == o.precision && top_uncompressed == o.top_uncompressed &&
           id_method == o.id_method && woodbury == o.woodbury && kappa == o.kappa && h == o.h && tol == o.tol;
  }
};

struct CacheLevel {
  int m = 0, k = 0, ring = 0, gr = 0;
  std::vector<int> sx, sy, piv;
  void *U = nullptr, *G = nullptr, *GL = nullptr, *GR = nullptr;
};

struct CacheEntry {
  CacheKey key;
  std::vector<CacheLevel> lev;  // levels 1..L (index 0 unused)
  double flops_compress = 0, flops_sibling = 0;
};

std::mutex g_cache_mu;
std::vector<CacheEntry>& cache() {
  static std::vector<CacheEntry> c;
  return c;
}

CacheKey key_of(const ls_handle* H) {
  CacheKey k;
  k.device = H->device;
  k.nx = H->grid.nx;
  k.ny = H->grid.ny;
  k.s = H->s;
  k.L = H->L;
  k.ring = H->ring;
  k.order_precond = H->opts.order_precond;
  k.precision = H->prec;
  k.top_uncompressed = H->opts.top_uncompressed;
  k.id_method = H->opts.id_method;
  k.woodbury = H->opts.woodbury;
  k.kappa = H->kappa;
  k.h = H->grid.h;
  k.tol = H->tol;
  return k;
}

// dst <- a new device copy of `bytes` bytes of src (nothing for 0 bytes)
int dup(void** dst, const void* src, size_t bytes, cudaStream_t st) {
  *dst = nullptr;
  if (bytes == 0 || !src) return LS_OK;
  int rc;
  if ((rc = dalloc(dst, bytes))) return rc;
  LS_CUDA_TRY(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyDeviceToDevice, st));
  return LS_OK;
}

void free_entry(CacheEntry& e) {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != e.key.device) cudaSetDevice(e.key.device);
  for (auto& l : e.lev) {
    for (void* p : {l.U, l.G, l.GL, l.GR})
      if (p) dfree(p);
  }
  e.lev.clear();
  if (cur != e.key.device) cudaSetDevice(cur);
}

}  // namespace

int cache_fetch(ls_handle* H, cudaStream_t st, bool* found) {
  *found = false;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  const CacheKey key = key_of(H);
  for (const CacheEntry& e : cache()) {
    if (!(e.key == key)) continue;
    const size_t es = elem_bytes(H);
    int rc;
    for (int l = 1; l <= H->L; ++l) {
      const CacheLevel& c = e.lev[l];
      LevelData& lv = H->lev[l];
      lv.m = c.m;
      lv.k = c.k;
      lv.ring = c.ring;
      lv.skel_x = c.sx;
      lv.skel_y = c.sy;
      lv.piv = c.piv;
      if ((rc = dup(&lv.U, c.U, es * (size_t)c.m * c.k, st))) return rc;
      if ((rc = dup(&lv.Gsib, c.G, es * (size_t)c.k * c.k, st))) return rc;
      lv.gr = c.gr;
      if (c.gr > 0) {
        if ((rc = dup(&lv.GL, c.GL, es * (size_t)c.k * c.gr, st))) return rc;
        if ((rc = dup(&lv.GR, c.GR, es * (size_t)c.k * c.gr, st))) return rc;
      }
      // a level of rank 0 still needs valid (empty) buffers
      if (!lv.U && (rc = dalloc(&lv.U, es))) return rc;
      if (!lv.Gsib && (rc = dalloc(&lv.Gsib, es))) return rc;
    }
    *found = true;
    return check_launch("compression cache fetch");
  }
  return LS_OK;
}

int cache_store(ls_handle* H, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  const CacheKey key = key_of(H);
  for (const CacheEntry& e : cache())
    if (e.key == key) return LS_OK;
  CacheEntry e;
  e.key = key;
  e.lev.resize(H->L + 1);
  const size_t es = elem_bytes(H);
  int rc = LS_OK;
  for (int l = 1; l <= H->L && !rc; ++l) {
    const LevelData& lv = H->lev[l];
    CacheLevel& c = e.lev[l];
    c.m = lv.m;
    c.k = lv.k;
    c.ring = lv.ring;
    c.gr = lv.gr;
    c.sx = lv.skel_x;
    c.sy = lv.skel_y;
    c.piv = lv.piv;
    if ((rc = dup(&c.U, lv.U, es * (size_t)lv.m * lv.k, st))) break;
    if ((rc = dup(&c.G, lv.Gsib, es * (size_t)lv.k * lv.k, st))) break;
    if (lv.gr > 0) {
      if ((rc = dup(&c.GL, lv.GL, es * (size_t)lv.k * lv.gr, st))) break;
      if ((rc = dup(&c.GR, lv.GR, es * (size_t)lv.k * lv.gr, st))) break;
    }
  }
  if (!rc) LS_CUDA_TRY(cudaStreamSynchronize(st));
  if (rc) {
    free_entry(e);
    return rc;
  }
  cache().push_back(std::move(e));
  return LS_OK;
}

// ------------------------------------------------------------- files
namespace {

constexpr char kMagic[8] = {'L', 'S', 'H', 'B', 'S', 'F', '0', '3'};

struct FileHeader {
  char magic[8];
  int header_bytes, opts_bytes, level_bytes;
  ls_grid grid;
  double kappa, tol;
  ls_opts opts;
  int L, s, ring, prec, nprob;
  double flops_build, flops_compress, flops_sibling, factor_bytes, probe_resid_max;
  int pivot_fallbacks;
};

struct FileLevel {
  int m, k, ring, gr, xr;
};

// sizes (entries) of a level's arrays
struct LevelSizes {
  size_t U, G, F, X, S;
};

LevelSizes level_sizes(const ls_handle* H, int l) {
  const LevelData& lv = H->lev[l];
  const size_t P = (size_t)H->nprob << l;
  const size_t n2 = l == H->L ? (size_t)H->s * H->s : 2 * (size_t)H->lev[l + 1].k;
  LevelSizes z;
  z.U = l >= 1 ? (size_t)lv.m * lv.k : 0;
  z.G = l >= 1 ? (size_t)lv.k * lv.k : 0;
  z.F = lv.gr > 0 ? (size_t)lv.k * lv.gr : 0;
  z.X = P * n2 * (lv.xr > 0 ? 2 * (size_t)lv.xr : n2);
  z.S = l >= 1 ? P * (size_t)lv.k * lv.k : 0;
  return z;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

// device <-> file through a pinned bounce buffer, in chunks
constexpr size_t kChunk = (size_t)8 << 20;

int write_dev(FILE* f, const void* d, size_t bytes, cudaStream_t st, void* bounce) {
  for (size_t o = 0; o < bytes; o += kChunk) {
    const size_t n = std::min(kChunk, bytes - o);
    LS_CUDA_TRY(cudaMemcpyAsync(bounce, static_cast<const char*>(d) + o, n, cudaMemcpyDeviceToHost, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
    if (fwrite(bounce, 1, n, f) != n) {
      set_last_error_text("ls_save: write failed");
      return LS_EINVAL;
    }
  }
  return LS_OK;
}

int read_dev(FILE* f, void* d, size_t bytes, cudaStream_t st, void* bounce) {
  for (size_t o = 0; o < bytes; o += kChunk) {
    const size_t n = std::min(kChunk, bytes - o);
    if (fread(bounce, 1, n, f) != n) {
      set_last_error_text("ls_load: file truncated");
      return LS_EINVAL;
    }
    LS_CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(d) + o, bounce, n, cudaMemcpyHostToDevice, st));
    LS_CUDA_TRY(cudaStreamSynchronize(st));
  }
  return LS_OK;
}

}  // namespace
}  // namespace ls

extern "C" {

void ls_compression_cache_clear(void) {
  std::lock_guard<std::mutex> lk(ls::g_cache_mu);
  for (auto& e : ls::cache()) ls::free_entry(e);
  ls::cache().clear();
}

int ls_save(const ls_handle* H, const char* path, void* stream) {
  if (!H || !path) return LS_EINVAL;
  if (int rc = ls::check_device(H)) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  ls::StreamScope scope(st);
  ls::File file;
  file.f = fopen(path, "wb");
  if (!file.f) {
    ls::set_last_error_text("ls_save: cannot open the file for writing");
    return LS_EINVAL;
  }
  ls::FileHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, ls::kMagic, 8);
  hd.header_bytes = sizeof(ls::FileHeader);
  hd.opts_bytes = sizeof(ls_opts);
  hd.level_bytes = sizeof(ls::FileLevel);
  hd.grid = H->grid;
  hd.kappa = H->kappa;
  hd.tol = H->tol;
  hd.opts = H->opts;
  hd.L = H->L;
  hd.s = H->s;
  hd.ring = H->ring;
  hd.prec = H->prec;
  hd.nprob = H->nprob;
  hd.flops_build = H->flops_build;
  hd.flops_compress = H->flops_compress;
  hd.flops_sibling = H->flops_sibling;
  hd.factor_bytes = H->factor_bytes;
  hd.probe_resid_max = H->probe_resid_max;
  hd.pivot_fallbacks = H->pivot_fallbacks;
  if (fwrite(&hd, sizeof(hd), 1, file.f) != 1) {
    ls::set_last_error_text("ls_save: write failed");
    return LS_EINVAL;
  }
  void* bounce = ls::pinned_scratch(ls::kChunk);
  if (!bounce) return LS_ENOMEM;
  const size_t es = ls::elem_bytes(H);
  const long long N = (long long)H->grid.nx * H->grid.ny * H->nprob;
  int rc;
  if ((rc = ls::write_dev(file.f, H->b, sizeof(double) * N, st, bounce))) return rc;
  // the level table and the skeletons, then every level's arrays (their sizes
  // depend on the next level's rank, so the loader reads the table first)
  for (int l = 0; l <= H->L; ++l) {
    const LevelData& lv = H->lev[l];
    ls::FileLevel fl{lv.m, lv.k, lv.ring, lv.gr, lv.xr};
    if (fwrite(&fl, sizeof(fl), 1, file.f) != 1) {
      ls::set_last_error_text("ls_save: write failed");
      return LS_EINVAL;
    }
  }
  for (int l = 1; l <= H->L; ++l) {
    const LevelData& lv = H->lev[l];
    if (lv.k > 0 && (fwrite(lv.skel_x.data(), sizeof(int), lv.k, file.f) != (size_t)lv.k ||
                     fwrite(lv.skel_y.data(), sizeof(int), lv.k, file.f) != (size_t)lv.k)) {
      ls::set_last_error_text("ls_save: write failed");
      return LS_EINVAL;
    }
  }
  for (int l = 0; l <= H->L; ++l) {
    const LevelData& lv = H->lev[l];
    const ls::LevelSizes z = ls::level_sizes(H, l);
    if ((rc = ls::write_dev(file.f, lv.U, es * z.U, st, bounce))) return rc;
    if ((rc = ls::write_dev(file.f, lv.Gsib, es * z.G, st, bounce))) return rc;
    if ((rc = ls::write_dev(file.f, lv.GL, es * z.F, st, bounce))) return rc;
    if ((rc = ls::write_dev(file.f, lv.GR, es * z.F, st, bounce))) return rc;
    if ((rc = ls::write_dev(file.f, lv.X, es * z.X, st, bounce))) return rc;
    if ((rc = ls::write_dev(file.f, lv.S, es * z.S, st, bounce))) return rc;
  }
  const size_t n = (size_t)H->s * H->s;
  if ((rc = ls::write_dev(file.f, H->XBU, es * ((size_t)H->nprob << H->L) * n * H->lev[H->L].k, st, bounce))) return rc;
  if (fflush(file.f) != 0) {
    ls::set_last_error_text("ls_save: write failed");
    return LS_EINVAL;
  }
  return LS_OK;
}

int ls_load(const char* path, void* stream, ls_handle** out) {
  if (!path || !out) return LS_EINVAL;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  ls::StreamScope scope(st);
  ls::File file;
  file.f = fopen(path, "rb");
  if (!file.f) {
    ls::set_last_error_text("ls_load: cannot open the file");
    return LS_EINVAL;
  }
  ls::FileHeader hd;
  if (fread(&hd, sizeof(hd), 1, file.f) != 1 || memcmp(hd.magic, ls::kMagic, 8) != 0 ||
      hd.header_bytes != (int)sizeof(ls::FileHeader) || hd.opts_bytes != (int)sizeof(ls_opts) ||
      hd.level_bytes != (int)sizeof(ls::FileLevel)) {
    ls::set_last_error_text("ls_load: not a file of ls_save (or of another version)");
    return LS_EINVAL;
  }
  const long long N = (long long)hd.grid.nx * hd.grid.ny * hd.nprob;
  if (hd.grid.nx < 2 || hd.grid.ny < 2 || hd.nprob < 1 || N > (1LL << 33)) {
    ls::set_last_error_text("ls_load: bad grid in the file");
    return LS_EINVAL;
  }
  std::vector<double> b((size_t)N);
  if (fread(b.data(), sizeof(double), (size_t)N, file.f) != (size_t)N) {
    ls::set_last_error_text("ls_load: file truncated");
    return LS_EINVAL;
  }
  ls_handle* H = new ls_handle();
  H->nprob = hd.nprob;
  auto fail = [&](int rc) {
    cudaStreamSynchronize(st);
    ls_free(H);
    return rc;
  };
  int rc = ls::setup_handle(H, &hd.grid, hd.kappa, b.data(), hd.tol, &hd.opts, st);
  if (rc) return fail(rc);
  if (H->L != hd.L || H->s != hd.s || H->ring != hd.ring || H->prec != hd.prec) {
    ls::set_last_error_text("ls_load: the file's tree does not match its grid and options");
    return fail(LS_EINVAL);
  }
  void* bounce = ls::pinned_scratch(ls::kChunk);
  if (!bounce) return fail(LS_ENOMEM);
  const size_t es = ls::elem_bytes(H);
  for (int l = 0; l <= H->L; ++l) {
    LevelData& lv = H->lev[l];
    ls::FileLevel fl;
    if (fread(&fl, sizeof(fl), 1, file.f) != 1) {
      ls::set_last_error_text("ls_load: file truncated");
      return fail(LS_EINVAL);
    }
    if (fl.k < 0 || fl.m < 0 || fl.gr > fl.k || fl.xr < 0 || (l >= 1 && fl.k > fl.m)) {
      ls::set_last_error_text("ls_load: bad level record");
      return fail(LS_EINVAL);
    }
    lv.m = fl.m;
    lv.k = fl.k;
    lv.ring = fl.ring;
    lv.gr = fl.gr;
    lv.xr = fl.xr;
  }
  for (int l = 1; l <= H->L; ++l) {
    LevelData& lv = H->lev[l];
    lv.skel_x.resize(lv.k);
    lv.skel_y.resize(lv.k);
    if (lv.k > 0 && (fread(lv.skel_x.data(), sizeof(int), lv.k, file.f) != (size_t)lv.k ||
                     fread(lv.skel_y.data(), sizeof(int), lv.k, file.f) != (size_t)lv.k)) {
      ls::set_last_error_text("ls_load: file truncated");
      return fail(LS_EINVAL);
    }
  }
  for (int l = 0; l <= H->L; ++l) {
    LevelData& lv = H->lev[l];
    const ls::LevelSizes z = ls::level_sizes(H, l);
    auto take = [&](void** p, size_t entries) -> int {
      if (entries == 0) return LS_OK;
      int r;
      if ((r = ls::dalloc(p, es * entries))) return r;
      return ls::read_dev(file.f, *p, es * entries, st, bounce);
    };
    if ((rc = take(&lv.U, z.U)) || (rc = take(&lv.Gsib, z.G)) || (rc = take(&lv.GL, z.F)) || (rc = take(&lv.GR, z.F)) ||
        (rc = take(&lv.X, z.X)) || (rc = take(&lv.S, z.S)))
      return fail(rc);
    if (l >= 1) {
      if (!lv.U && (rc = ls::dalloc(&lv.U, es))) return fail(rc);
      if (!lv.Gsib && (rc = ls::dalloc(&lv.Gsib, es))) return fail(rc);
    }
  }
  {
    const size_t n = (size_t)H->s * H->s, e = ((size_t)H->nprob << H->L) * n * H->lev[H->L].k;
    if ((rc = ls::dalloc(&H->XBU, es * std::max<size_t>(e, 1)))) return fail(rc);
    if (e && (rc = ls::read_dev(file.f, H->XBU, es * e, st, bounce))) return fail(rc);
  }
  H->flops_build = hd.flops_build;
  H->flops_compress = hd.flops_compress;
  H->flops_sibling = hd.flops_sibling;
  H->factor_bytes = hd.factor_bytes;
  H->probe_resid_max = hd.probe_resid_max;
  H->pivot_fallbacks = hd.pivot_fallbacks;
  H->compression_reused = 1;
  if ((rc = ls::hbs_finish(H, st))) return fail(rc);
  LS_CUDA_TRY(cudaStreamSynchronize(st));
  *out = H;
  return LS_OK;
}

}  // extern "C"
