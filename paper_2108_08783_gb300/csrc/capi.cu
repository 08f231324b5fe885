// C ABI of the library (declared in include/lbm.h): context lifetime, device
// memory, host<->device copies and kernel launches.  Every step of the method
// runs in the kernels of kernels.cu; this file only marshals.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

#ifndef LBM_SIDE_PRIORITY
#define LBM_SIDE_PRIORITY 1
#endif
// L2 prefetch distance of the bulk kernel (tiles ahead) by storage, measured on
// GB300: FP32 gains from prefetching 4096 tiles ahead; the 16-bit storages are
// issue-bound and lose more to the prefetch instructions than they gain; FP64
// is ALU-bound either way.  -DLBM_DEFAULT_PREFETCH=n overrides.
// Bulk kernel mode (LBM_TUNE_BULK_SITES) by storage, measured on GB300: the
// 16-bit storages gain from two sites per lane, adjacent sites on even steps
// and two tiles on odd steps (+11-15 % on the long tube, +4 % on the tree,
// +9 % on the 256-tube ensemble); FP32 is DRAM-bound with one site per lane
// and loses 0-6 % with two; FP64 has one form only.
// -DLBM_DEFAULT_BULK_SITES=n overrides.
inline int32_t default_bulk_sites(int storage) {
#ifdef LBM_DEFAULT_BULK_SITES
  (void)storage;
  return LBM_DEFAULT_BULK_SITES;
#else
  return (storage == LBM_F16S || storage == LBM_BF16S) ? 2 : 1;
#endif
}

inline int64_t default_prefetch(int storage) {
#ifdef LBM_DEFAULT_PREFETCH
  (void)storage;
  return LBM_DEFAULT_PREFETCH;
#else
  return storage == LBM_F32 ? 4096 : 0;
#endif
}

using lbm::DevLattice;
using lbm::HostLattice;

struct lbm_ctx {
  HostLattice L;
  std::vector<lbm_iolet> iolets;
  int storage = LBM_F64;
  double tau = 1.0;
  int wall_model = LBM_WALL_BOUNCEBACK;
  double rho0 = 1.0;
  int64_t step = 0;
  cudaStream_t stream = nullptr;
  lbm_allocator alloc{};
  bool user_alloc = false;
  std::vector<void*> owned;
  size_t dev_bytes = 0;
  DevLattice d;
  int64_t* iolet_off = nullptr;
  int64_t* iolet_sites = nullptr;
  double* partial = nullptr;
  double* red_out = nullptr;
  std::string err;
  int64_t prefetch = 0;  // L2 prefetch distance (tiles), set from the storage at build
  int32_t bulk_sites = 1;  // bulk kernel mode, set from the storage at build
  int32_t bulk_warps = 4;  // warps per CTA of the bulk kernel
  int32_t n_sms = 0;       // SMs of the context's device
  // captured steps (LBM_TUNE_GRAPH_STEPS): G steps replayed as one CUDA graph
  // on a private stream, ordered with the context's stream by events; the
  // inlet phase reads a device step counter that the graph advances
  int64_t graph_steps = 0;
  cudaStream_t gstream = nullptr;
  cudaEvent_t g_in = nullptr, g_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int gexec_parity = -1;
  int64_t gexec_steps = 0;
  // device step counter: holds the even floor of the step it was last made
  // right for (step_d_for; -1: unknown); the captured kernels add it to their
  // compile-time offset (the parity plus the step within the block)
  int64_t* step_d = nullptr;
  int64_t step_d_for = -1;
  // tensor map of the populations as a [19][npad] array of 16-bit elements,
  // boxes of 32 x 19 (staged-row bulk kernel), made on first use
  alignas(64) CUtensorMap tmap;
  bool tmap_ready = false;
  // optional per-kernel timing (lbm_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev;  // 3 per profiled step
  // side stream of the boundary kernel, and the fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  size_t ev_used = 0;
  int32_t* coords_dev = nullptr;  // [n][3] voxel coordinates, uploaded on first use (warm start)
  // fused diagnostics (lbm_step_diag), set up on first use: kDiagSets sets
  // of buffers used in turn, so that the final sums and the copy to the host
  // of one diagnostic step run on their own (high-priority) stream beside the
  // next steps
  static constexpr int kDiagSets = 4;
  bool diag_ready = false;
  double* diag_mass[kDiagSets] = {};
  double* diag_j[kDiagSets] = {};
  double* diag_part[kDiagSets] = {};
  unsigned* diag_done[kDiagSets] = {};
  double* diag_out[kDiagSets] = {};
  int64_t* diag_io_off = nullptr;
  int64_t* diag_io_q = nullptr;
  int diag_fpi = 1;  // final-sum blocks per iolet
  cudaStream_t diag_stream = nullptr;
  cudaEvent_t diag_filled[kDiagSets] = {};  // main stream: the step kernels wrote set b
  cudaEvent_t diag_free[kDiagSets] = {};    // diagnostic stream: set b copied out
  bool diag_used[kDiagSets] = {};
  int64_t diag_seq = 0;
};

namespace {

// Steps per captured graph of a lattice by default: +3 % on the long tube
// against direct launches (100 gains another 0.1-0.4 %).
constexpr int64_t kDefaultGraphSteps = 20;

constexpr uint64_t kCkptMagic = 0x314b43504d424cULL;  // "LBMPCK1"

// Message of the last failed lbm_build_lattice on this thread (no context exists then).
thread_local std::string g_build_err;

int fail(lbm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return fail(c, LBM_ECUDA, buf);
}

void* dev_alloc_raw(lbm_ctx* c, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (c->user_alloc) {
    p = c->alloc.alloc(bytes, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dev_free_raw(lbm_ctx* c, void* p) {
  if (!p) return;
  if (c->user_alloc) c->alloc.free(p, c->alloc.user);
  else cudaFree(p);
}

// Owned allocation, released by lbm_destroy.
template <class T>
T* dev_alloc(lbm_ctx* c, size_t count) {
  void* p = dev_alloc_raw(c, count * sizeof(T));
  if (p) {
    c->owned.push_back(p);
    c->dev_bytes += (count * sizeof(T) + 255) & ~(size_t)255;
  }
  return static_cast<T*>(p);
}

// Temporary allocation freed when it goes out of scope (after a stream sync).
struct Temp {
  lbm_ctx* c;
  void* p = nullptr;
  Temp(lbm_ctx* c_, size_t bytes) : c(c_) { p = bytes ? dev_alloc_raw(c, bytes) : nullptr; }
  ~Temp() { dev_free_raw(c, p); }
};

template <class T>
cudaError_t h2d(lbm_ctx* c, T* dst, const T* src, size_t count) {
  if (count == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, c->stream);
}

int check_launch(lbm_ctx* c, int rc, const char* what) {
  if (rc != 0) return cuda_fail(c, (cudaError_t)rc, what);
  return LBM_OK;
}

int sync(lbm_ctx* c, const char* what) {
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && c->diag_stream) e = cudaStreamSynchronize(c->diag_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  return LBM_OK;
}

bool odd_layout(const lbm_ctx* c) { return (c->step & 1) != 0; }

}  // namespace

extern "C" {

const char* lbm_status_string(int s) {
  switch (s) {
    case LBM_OK: return "LBM_OK";
    case LBM_EINVAL: return "LBM_EINVAL";
    case LBM_ENOMEM: return "LBM_ENOMEM";
    case LBM_ECUDA: return "LBM_ECUDA";
    case LBM_EUNSTABLE: return "LBM_EUNSTABLE";
    case LBM_ETIMEOUT: return "LBM_ETIMEOUT";
    case LBM_ESTATE: return "LBM_ESTATE";
    case LBM_ECHECK: return "LBM_ECHECK";
  }
  return "LBM_E?";
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : g_build_err.c_str(); }

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->diag_stream) cudaStreamSynchronize(c->diag_stream);
  if (c->gstream) cudaStreamSynchronize(c->gstream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->g_in) cudaEventDestroy(c->g_in);
  if (c->g_out) cudaEventDestroy(c->g_out);
  if (c->gstream) cudaStreamDestroy(c->gstream);
  for (void* p : c->owned) dev_free_raw(c, p);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->join) cudaEventDestroy(c->join);
  if (c->side) cudaStreamDestroy(c->side);
  for (int b = 0; b < lbm_ctx::kDiagSets; ++b) {
    if (c->diag_filled[b]) cudaEventDestroy(c->diag_filled[b]);
    if (c->diag_free[b]) cudaEventDestroy(c->diag_free[b]);
  }
  if (c->diag_stream) cudaStreamDestroy(c->diag_stream);
  delete c;
}

int lbm_profile(lbm_ctx* c, int32_t enable) {
  if (!c) return LBM_EINVAL;
  c->prof = enable != 0;
  c->ev_used = 0;
  return LBM_OK;
}

int lbm_profile_read(lbm_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return LBM_EINVAL;
  int rc = sync(c, "lbm_profile_read");
  if (rc != LBM_OK) return rc;
  ms[0] = ms[1] = 0.0;
  launches[0] = launches[1] = 0;
  for (size_t k = 0; k + 2 < c->ev_used; k += 3) {
    float a = 0.f, b = 0.f;
    cudaError_t e = cudaEventElapsedTime(&a, c->ev[k], c->ev[k + 2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, c->ev[k], c->ev[k + 1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_profile_read");
    ms[0] += a;
    ms[1] += b;
    launches[0] += c->d.n_tiles > c->d.n_boundary;
    launches[1] += c->d.n_boundary > 0;
  }
  c->ev_used = 0;
  return LBM_OK;
}

int lbm_build_lattice(const uint8_t* labels, int32_t nx, int32_t ny, int32_t nz,
                      const lbm_iolet* iolets, int32_t n_iolets, int32_t storage, double tau,
                      const lbm_allocator* alloc, void* cuda_stream, lbm_ctx** out) {
  g_build_err.clear();
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (storage < LBM_F64 || storage > LBM_BF16S) {
    g_build_err = "unknown storage";
    return LBM_EINVAL;
  }
  if (alloc && (!alloc->alloc || !alloc->free)) {
    g_build_err = "allocator needs both alloc and free";
    return LBM_EINVAL;
  }
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  c->storage = storage;
  c->prefetch = default_prefetch(storage);
  c->bulk_sites = default_bulk_sites(storage);
  c->graph_steps = kDefaultGraphSteps;
  c->tau = tau;
  c->stream = (cudaStream_t)cuda_stream;
  if (alloc) {
    c->alloc = *alloc;
    c->user_alloc = true;
  }
  int rc;
  try {
    rc = lbm::build_lattice(labels, nx, ny, nz, iolets, n_iolets, tau, c->L, c->err);
  } catch (const std::bad_alloc&) {
    rc = LBM_ENOMEM;
  }
  if (rc != LBM_OK) {
    g_build_err = rc == LBM_ENOMEM ? std::string("host allocation failed") : c->err;
    delete c;
    return rc;
  }
  c->iolets.assign(iolets, iolets + n_iolets);
  HostLattice& L = c->L;
  DevLattice& d = c->d;
  d.n = L.n;
  // slack past the last site: the step kernel copies 16-byte-aligned runs of
  // 32 + 16/sizeof(storage) elements that may reach up to 8 elements beyond it
  d.npad = ((L.n + 64 + 127) / 128) * 128;
  d.n_tiles = L.n_tiles;
  d.n_boundary = L.n_uniform + L.n_irregular;
  d.slot_stride = L.n_slots;
  d.n_iolets = n_iolets;
  const size_t S = (size_t)L.n_slots;
  const size_t sz = lbm::storage_bytes(storage);
  d.pop = dev_alloc<unsigned char>(c, (size_t)lbm::kQ * d.npad * sz);
  lbm::TileDesc* td = dev_alloc<lbm::TileDesc>(c, L.tiles.size());
  lbm::LaunchDesc* to = dev_alloc<lbm::LaunchDesc>(c, L.launch.size());
  uint32_t* sm = dev_alloc<uint32_t>(c, S);
  uint32_t* sio = dev_alloc<uint32_t>(c, S);
  int32_t* sn = dev_alloc<int32_t>(c, 18 * S);
  // inlet profile and wall F in the compute type (FP64 storage: double; the
  // FP32-compute storages: float, so the step kernels convert nothing)
  const size_t cb = storage == LBM_F64 ? sizeof(double) : sizeof(float);
  unsigned char* sp = dev_alloc<unsigned char>(c, 3 * S * cb);
  unsigned char* sF = dev_alloc<unsigned char>(c, S * cb);
  double* sK = dev_alloc<double>(c, S);
  double* sdE = dev_alloc<double>(c, S);
  double* sUw = dev_alloc<double>(c, 3 * S);
  lbm::IoletDev* io = dev_alloc<lbm::IoletDev>(c, n_iolets);
  int* err = dev_alloc<int>(c, 1);
  c->iolet_off = dev_alloc<int64_t>(c, L.iolet_off.size());
  c->iolet_sites = dev_alloc<int64_t>(c, L.iolet_sites.size());
  c->partial = dev_alloc<double>(c, lbm::reduce_partials());
  c->red_out = dev_alloc<double>(c, 1 + n_iolets);
  int32_t* mt = L.multi_tiles.empty() ? nullptr : dev_alloc<int32_t>(c, L.multi_tiles.size());
  int32_t* stab = L.seg_tab.empty() ? nullptr : dev_alloc<int32_t>(c, L.seg_tab.size());
  if (!d.pop || !td || !to || !sm || !sio || !sn || !sp || !sF || !sK || !sdE || !sUw ||
      !io || !err || !c->iolet_off || !c->iolet_sites || !c->partial || !c->red_out ||
      (!L.multi_tiles.empty() && !mt) || (!L.seg_tab.empty() && !stab)) {
    g_build_err = "device allocation failed";
    lbm_destroy(c);
    return LBM_ENOMEM;
  }
  d.tiles = td;
  d.launch = to;
  d.slot_mask = sm;
  d.slot_io = sio;
  d.slot_nbr = sn;
  d.slot_prof = sp;
  d.slot_F = sF;
  d.slot_kappa = sK;
  d.slot_dE = sdE;
  d.slot_Uw = sUw;
  d.iolets = io;
  d.err = err;
  d.multi_tiles = mt;
  d.seg_tab = stab;
  d.n_multi = (int64_t)L.multi_tiles.size();
#ifdef LBM_CHECKED
  // checked builds: per-slot store counts of the current step
  d.chk = dev_alloc<int>(c, (size_t)lbm::kQ * d.npad);
  if (!d.chk) {
    g_build_err = "device allocation failed";
    lbm_destroy(c);
    return LBM_ENOMEM;
  }
  if (cudaMemsetAsync(d.chk, 0, (size_t)lbm::kQ * d.npad * sizeof(int), c->stream) != cudaSuccess) {
    g_build_err = "checked build: count reset failed";
    lbm_destroy(c);
    return LBM_ECUDA;
  }
#endif
  std::vector<lbm::IoletDev> hio(n_iolets);
  for (int k = 0; k < n_iolets; ++k) {
    const lbm_iolet& s = iolets[k];
    lbm::IoletDev& t = hio[k];
    std::memset(&t, 0, sizeof t);
    t.kind = s.kind;
    t.steady = s.period > 0.0 ? 0 : 1;
    t.rho = s.rho;
    t.u_mean = s.u_mean;
    t.u_amp = s.u_amp;
    t.period = s.period > 0.0 ? s.period : 1.0;
    t.phase = s.phase;
    const double an = std::sqrt(s.axis[0] * s.axis[0] + s.axis[1] * s.axis[1] + s.axis[2] * s.axis[2]);
    for (int a = 0; a < 3; ++a) t.axis[a] = s.axis[a] / an;
    // fixed-point phase (fraction of a period, units of 2^-64)
    const double inv = 1.0 / t.period;
    t.phase_inc = lbm::frac_to_u64(inv - std::floor(inv));
    const double ph = t.phase * (0.5 / M_PI);
    t.phase_off = lbm::frac_to_u64(ph - std::floor(ph));
    t.rho_f = (float)t.rho;
    t.drho_f = (float)(t.rho - 1.0);
    t.u_mean_f = (float)t.u_mean;
    t.u_amp_f = (float)t.u_amp;
    for (int a = 0; a < 3; ++a) t.axis_f[a] = (float)t.axis[a];
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(h2d(c, td, L.tiles.data(), L.tiles.size()));
  chk(h2d(c, to, L.launch.data(), L.launch.size()));
  chk(h2d(c, sm, L.slot_mask.data(), S));
  chk(h2d(c, sio, L.slot_io.data(), S));
  chk(h2d(c, sn, L.slot_nbr.data(), 18 * S));
  std::vector<float> prof_f;
  if (storage == LBM_F64) {
    chk(h2d(c, reinterpret_cast<double*>(sp), L.slot_prof.data(), 3 * S));
  } else {
    prof_f.assign(L.slot_prof.begin(), L.slot_prof.end());  // rounded once, here
    chk(h2d(c, reinterpret_cast<float*>(sp), prof_f.data(), 3 * S));
  }
  chk(h2d(c, io, hio.data(), hio.size()));
  chk(h2d(c, c->iolet_off, L.iolet_off.data(), L.iolet_off.size()));
  chk(h2d(c, c->iolet_sites, L.iolet_sites.data(), L.iolet_sites.size()));
  if (mt) chk(h2d(c, mt, L.multi_tiles.data(), L.multi_tiles.size()));
  if (stab) chk(h2d(c, stab, L.seg_tab.data(), L.seg_tab.size()));
  if (S) {
    chk(cudaMemsetAsync(sF, 0, S * cb, c->stream));
    chk(cudaMemsetAsync(sK, 0, S * sizeof(double), c->stream));
    chk(cudaMemsetAsync(sdE, 0, S * sizeof(double), c->stream));
    chk(cudaMemsetAsync(sUw, 0, 3 * S * sizeof(double), c->stream));
  }
  chk(cudaMemsetAsync(err, 0, sizeof(int), c->stream));
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      c->n_sms = sms;
    cudaGetLastError();
  }
  chk(cudaMemsetAsync(d.pop, 0, (size_t)lbm::kQ * d.npad * sz, c->stream));
  if (e != cudaSuccess) {
    rc = cuda_fail(c, e, "lbm_build_lattice upload");
    g_build_err = c->err;
    lbm_destroy(c);
    return rc;
  }
  {
    // side stream and fork/join events of the boundary kernel
    // higher priority, so that the block scheduler dispatches boundary CTAs
    // as soon as bulk CTAs retire instead of after the whole bulk grid
    int lo = 0, hi = 0;
    cudaError_t ge = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (ge == cudaSuccess)
      ge = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, LBM_SIDE_PRIORITY ? hi : lo);
    if (ge == cudaSuccess) ge = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (ge == cudaSuccess) ge = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    if (ge != cudaSuccess) {
      rc = cuda_fail(c, ge, "side stream");
      g_build_err = c->err;
      lbm_destroy(c);
      return rc;
    }
  }
  rc = check_launch(c, lbm::launch_init(storage, d, nullptr, nullptr, c->stream), "init kernel");
  if (rc == LBM_OK) rc = sync(c, "lbm_build_lattice");
  if (rc != LBM_OK) {
    g_build_err = c->err;
    lbm_destroy(c);
    return rc;
  }
  *out = c;
  return LBM_OK;
}

int lbm_set_stream(lbm_ctx* c, void* s) {
  if (!c) return LBM_EINVAL;
  c->stream = (cudaStream_t)s;
  return LBM_OK;
}

int lbm_set_wall_params(lbm_ctx* c, int32_t wall_model, double rho0, const double* F,
                        const double* kappa, int64_t n) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  if (wall_model != LBM_WALL_BOUNCEBACK && wall_model != LBM_WALL_ELASTIC_GZS)
    return fail(c, LBM_EINVAL, "unknown wall model");
  if (!std::isfinite(rho0)) return fail(c, LBM_EINVAL, "rho0 must be finite");
  const int64_t W = (int64_t)c->L.wall_sites.size();
  if (W > 0 && n != 1 && n != W) return fail(c, LBM_EINVAL, "n must be 1 or n_wall_sites");
  const size_t S = (size_t)c->L.n_slots;
  std::vector<double> hF(S, 0.0), hK(S, 0.0);
  for (int64_t w = 0; w < W; ++w) {
    const double f = F ? F[n == 1 ? 0 : w] : 0.0;
    const double k = kappa ? kappa[n == 1 ? 0 : w] : 0.0;
    if (!std::isfinite(f) || !std::isfinite(k) || f < 0.0 || k < 0.0)
      return fail(c, LBM_EINVAL, "F and kappa must be finite and >= 0");
    hF[c->L.wall_slot[w]] = f;
    hK[c->L.wall_slot[w]] = k / 3.0;  // the kernel applies kappa c_s^2 to (rho - rho0)
  }
  cudaError_t e;
  std::vector<float> hF_f;
  if (c->storage == LBM_F64) {
    e = h2d(c, static_cast<double*>(const_cast<void*>(c->d.slot_F)), hF.data(), S);
  } else {
    hF_f.assign(hF.begin(), hF.end());
    e = h2d(c, static_cast<float*>(const_cast<void*>(c->d.slot_F)), hF_f.data(), S);
  }
  if (e == cudaSuccess) e = h2d(c, const_cast<double*>(c->d.slot_kappa), hK.data(), S);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_wall_params");
  int rc = sync(c, "lbm_set_wall_params");
  if (rc != LBM_OK) return rc;
  c->wall_model = wall_model;
  c->rho0 = rho0;
  c->gexec_steps = 0;  // a captured step graph holds the old wall constants
  return LBM_OK;
}

int lbm_init_fields(lbm_ctx* c, const double* rho, const double* u) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  const size_t n = (size_t)c->L.n;
  Temp tr(c, rho ? n * sizeof(double) : 0), tu(c, u ? 3 * n * sizeof(double) : 0);
  if ((rho && !tr.p) || (u && !tu.p)) return fail(c, LBM_ENOMEM, "lbm_init_fields: allocation");
  cudaError_t e = cudaSuccess;
  if (rho) e = h2d(c, (double*)tr.p, rho, n);
  if (u && e == cudaSuccess) e = h2d(c, (double*)tu.p, u, 3 * n);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_init_fields copy");
  int rc = check_launch(c, lbm::launch_init(c->storage, c->d, rho ? (double*)tr.p : nullptr,
                                            u ? (double*)tu.p : nullptr, c->stream),
                        "init kernel");
  if (rc == LBM_OK) rc = sync(c, "lbm_init_fields");
  if (rc == LBM_OK) c->step = 0;
  return rc;
}

namespace {

// The populations as a 2-D tensor for TMA copies: [19 rows][npad] 16-bit
// elements (row stride npad elements), boxes of one tile (32) x 19 rows.
int make_tmap(lbm_ctx* c) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q{};
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess)
    return fail(c, LBM_ECUDA, "staged rows: no cuTensorMapEncodeTiled");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  const cuuint64_t dims[2] = {(cuuint64_t)c->d.npad, (cuuint64_t)lbm::kQ};
  const cuuint64_t strides[1] = {(cuuint64_t)c->d.npad * 2};
  const cuuint32_t box[2] = {(cuuint32_t)lbm::kTile, (cuuint32_t)lbm::kQ};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(&c->tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, c->d.pop, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, LBM_ECUDA, "staged rows: tensor map encoding failed");
  c->tmap_ready = true;
  return LBM_OK;
}

// n_steps timesteps; with diag_last the last one also writes the fused
// diagnostics of the state it reads.
void drop_graph(lbm_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gexec_parity = -1;
  c->gexec_steps = 0;
}

// The launch parameters of the context's steps (the step index set per step).
lbm::StepParams step_params(const lbm_ctx* c) {
  lbm::StepParams p{};
  p.rho0 = c->rho0;
  p.rho0_f = (float)c->rho0;
  p.rho0_exact = (double)p.rho0_f == c->rho0 ? 1 : 0;
  p.omega = 1.0 / c->tau;
  p.omega_f = (float)p.omega;
  p.elastic = c->wall_model == LBM_WALL_ELASTIC_GZS ? 1 : 0;
  p.prefetch = c->prefetch;
  p.step_dev = nullptr;
  p.bulk_sites = c->bulk_sites;
  p.bulk_warps = c->bulk_warps;
  p.n_sms = c->n_sms;
  p.tmap = c->tmap_ready ? &c->tmap : nullptr;
  return p;
}

int run_steps(lbm_ctx* c, int64_t n_steps, bool diag_last) {
  lbm::StepParams p = step_params(c);
#ifndef LBM_CHECKED
  const int64_t G = c->graph_steps;
  if (G > 0 && n_steps >= G && !diag_last && !c->prof) {
    // whole blocks of G steps as graph replays on the private stream
    cudaError_t r = cudaSuccess;
    if (!c->gstream) r = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking);
    if (r == cudaSuccess && !c->g_in) r = cudaEventCreateWithFlags(&c->g_in, cudaEventDisableTiming);
    if (r == cudaSuccess && !c->g_out) r = cudaEventCreateWithFlags(&c->g_out, cudaEventDisableTiming);
    if (r != cudaSuccess) return cuda_fail(c, r, "graph stream");
    if (!c->step_d) {
      c->step_d = dev_alloc<int64_t>(c, 1);
      if (!c->step_d) return fail(c, LBM_ENOMEM, "graph step counter");
    }
    r = cudaEventRecord(c->g_in, c->stream);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(c->gstream, c->g_in, 0);
    if (r != cudaSuccess) return cuda_fail(c, r, "graph ordering");
    const lbm::StepStreams gs{c->gstream, c->side, c->fork, c->join};
    const int parity = (int)(c->step & 1);
    if (!c->gexec || c->gexec_parity != parity || c->gexec_steps != G) {
      drop_graph(c);
      cudaGraph_t graph = nullptr;
      r = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
      for (int64_t s = 0; s < G && r == cudaSuccess; ++s) {
        p.step = parity + s;  // the kernels add *step_d = step - parity
        p.step_dev = c->step_d;
        p.write_state = s == G - 1 ? 1 : 0;
        const int lr = lbm::launch_step(c->storage, c->d, p, gs, nullptr);
        if (lr != 0) r = (cudaError_t)lr;
      }
      if (r == cudaSuccess) r = (cudaError_t)lbm::launch_advance(c->step_d, G, c->gstream);
      cudaError_t r2 = cudaStreamEndCapture(c->gstream, &graph);
      if (r == cudaSuccess) r = r2;
      if (r == cudaSuccess) r = cudaGraphInstantiate(&c->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (r != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_fail(c, r, "step graph capture");
      }
      c->gexec_parity = parity;
      c->gexec_steps = G;
    }
    if (c->step_d_for != c->step)
      r = (cudaError_t)lbm::launch_set_step(c->step_d, c->step - parity, c->gstream);
    int64_t done = 0;
    for (; r == cudaSuccess && n_steps - done >= G; done += G) r = cudaGraphLaunch(c->gexec, c->gstream);
    if (r != cudaSuccess) return cuda_fail(c, r, "step graph launch");
    c->step += done;
    c->step_d_for = c->step;  // each replay advanced the counter by G
    p.step_dev = nullptr;
    for (int64_t s = done; s < n_steps; ++s) {
      p.step = c->step;
      p.write_state = s == n_steps - 1 ? 1 : 0;
      p.diag = 0;
      const int lr = lbm::launch_step(c->storage, c->d, p, gs, nullptr);
      if (lr != 0) return cuda_fail(c, (cudaError_t)lr, "step kernels");
      ++c->step;
    }
    r = cudaEventRecord(c->g_out, c->gstream);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(c->stream, c->g_out, 0);
    if (r != cudaSuccess) return cuda_fail(c, r, "graph ordering");
    return LBM_OK;
  }
#endif
  for (int64_t s = 0; s < n_steps; ++s) {
    p.step = c->step;
    p.write_state = s == n_steps - 1 ? 1 : 0;
    p.diag = diag_last && s == n_steps - 1 ? 1 : 0;
    void* ev[3] = {nullptr, nullptr, nullptr};
    if (c->prof) {
      while (c->ev.size() < c->ev_used + 3) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return cuda_fail(c, r, "lbm_step event");
        c->ev.push_back(e);
      }
      for (int k = 0; k < 3; ++k) ev[k] = c->ev[c->ev_used + k];
      c->ev_used += 3;
    }
    const lbm::StepStreams ss{c->stream, c->side, c->fork, c->join};
    int rc = lbm::launch_step(c->storage, c->d, p, ss, c->prof ? ev : nullptr);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "step kernels");
#ifdef LBM_CHECKED
    rc = lbm::launch_check_counts(c->d, c->stream);
    if (rc != 0) return cuda_fail(c, (cudaError_t)rc, "checked build: count kernel");
#endif
    ++c->step;
  }
  return LBM_OK;
}

// Device tables of the fused diagnostics: the boundary tiles with sites
// linked to iolets numbered in launch order, and per iolet the places of its
// sites among those tiles' lanes.
int diag_setup(lbm_ctx* c) {
  if (c->diag_ready) return LBM_OK;
  const HostLattice& L = c->L;
  const int64_t nb = c->d.n_boundary;
  const int nio = (int)c->iolets.size();
  std::vector<int32_t> iotile((size_t)nb, -1);
  int32_t n_io = 0;
  for (int64_t k = 0; k < nb; ++k) {
    bool any = false;
    for (int l = 0; l < lbm::kTile; ++l) {
      const size_t sl = (size_t)k * lbm::kTile + l;
      if ((L.slot_io[sl] & lbm::kDirBits) || (L.slot_mask[sl] & lbm::kMultiIolet)) any = true;
    }
    if (any) iotile[(size_t)k] = n_io++;
  }
  std::vector<int64_t> ioff((size_t)nio + 1, 0), q;
  for (int k = 0; k < nio; ++k) {
    for (int64_t i = L.iolet_off[k]; i < L.iolet_off[k + 1]; ++i) {
      const int64_t x = L.iolet_sites[(size_t)i];
      const int32_t slot0 = L.tiles[(size_t)(x / lbm::kTile)].slot;
      const int32_t it = slot0 >= 0 ? iotile[(size_t)(slot0 / lbm::kTile)] : -1;
      if (it < 0) return fail(c, LBM_ESTATE, "diagnostics: an iolet site outside the iolet tiles");
      q.push_back((int64_t)it * lbm::kTile + x % lbm::kTile);
    }
    ioff[(size_t)k + 1] = (int64_t)q.size();
  }
  const int64_t js = (int64_t)(n_io > 0 ? n_io : 1) * lbm::kTile;
  int64_t max_sites = 0;
  for (int k = 0; k < nio; ++k) max_sites = std::max(max_sites, ioff[(size_t)k + 1] - ioff[(size_t)k]);
  c->diag_fpi = lbm::diag_flux_blocks(max_sites);
  int32_t* it_d = dev_alloc<int32_t>(c, nb > 0 ? (size_t)nb : 1);
  c->diag_io_off = dev_alloc<int64_t>(c, ioff.size());
  c->diag_io_q = dev_alloc<int64_t>(c, q.empty() ? 1 : q.size());
  bool ok = it_d && c->diag_io_off && c->diag_io_q;
  for (int b = 0; b < lbm_ctx::kDiagSets; ++b) {
    c->diag_mass[b] = dev_alloc<double>(c, (size_t)c->d.n_tiles);
    c->diag_j[b] = dev_alloc<double>(c, 3 * (size_t)js);
    c->diag_part[b] = dev_alloc<double>(c, (size_t)lbm::diag_blocks(nio, c->diag_fpi));
    c->diag_done[b] = dev_alloc<unsigned>(c, 1);
    c->diag_out[b] = dev_alloc<double>(c, 1 + (size_t)nio);
    ok = ok && c->diag_mass[b] && c->diag_j[b] && c->diag_part[b] && c->diag_done[b] &&
         c->diag_out[b];
  }
  if (!ok) return fail(c, LBM_ENOMEM, "diagnostics: device allocation");
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
  chk(h2d(c, it_d, iotile.data(), iotile.size()));
  chk(h2d(c, c->diag_io_off, ioff.data(), ioff.size()));
  chk(h2d(c, c->diag_io_q, q.data(), q.size()));
  for (int b = 0; b < lbm_ctx::kDiagSets; ++b) {
    chk(cudaMemsetAsync(c->diag_done[b], 0, sizeof(unsigned), c->stream));
    chk(cudaMemsetAsync(c->diag_mass[b], 0, (size_t)c->d.n_tiles * sizeof(double), c->stream));
    chk(cudaMemsetAsync(c->diag_j[b], 0, 3 * (size_t)js * sizeof(double), c->stream));
  }
  if (e == cudaSuccess && !c->diag_stream) {
    // highest priority: its few blocks start ahead of the next bulk kernel's
    int lo = 0, hi = 0;
    e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&c->diag_stream, cudaStreamNonBlocking, hi);
  }
  for (int b = 0; b < lbm_ctx::kDiagSets && e == cudaSuccess; ++b) {
    if (!c->diag_filled[b]) e = cudaEventCreateWithFlags(&c->diag_filled[b], cudaEventDisableTiming);
    if (e == cudaSuccess && !c->diag_free[b])
      e = cudaEventCreateWithFlags(&c->diag_free[b], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "diagnostics setup");
  int rc = sync(c, "diagnostics setup");  // the host tables are temporaries
  if (rc != LBM_OK) return rc;
  c->d.diag_iotile = it_d;
  c->d.diag_jstride = js;
  c->diag_ready = true;
  return LBM_OK;
}

}  // namespace

int lbm_step(lbm_ctx* c, int64_t n_steps) {
  if (!c) return LBM_EINVAL;
  if (n_steps < 0) return fail(c, LBM_EINVAL, "n_steps must be >= 0");
  return run_steps(c, n_steps, false);
}

int lbm_step_diag(lbm_ctx* c, int64_t n_steps, double* out) {
  if (!c || !out) return LBM_EINVAL;
  c->err.clear();
  if (n_steps < 1) return fail(c, LBM_EINVAL, "n_steps must be >= 1");
  int rc = diag_setup(c);
  if (rc != LBM_OK) return rc;
  // buffer set b: its previous final sums and copy are done before the step
  // kernels write it again (normally long since)
  const int b = (int)(c->diag_seq % lbm_ctx::kDiagSets);
  cudaError_t e = cudaSuccess;
  c->d.diag_mass = c->diag_mass[b];
  c->d.diag_j = c->diag_j[b];
  // (a captured graph per diagnostic step measured no faster: the stream
  // hops around it cost what the launches save)
  if (n_steps > 1) {
    rc = run_steps(c, n_steps - 1, false);  // captured graphs where they apply
    if (rc != LBM_OK) return rc;
  }
  if (c->diag_used[b]) e = cudaStreamWaitEvent(c->stream, c->diag_free[b], 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_diag order");
  rc = run_steps(c, 1, true);
  if (rc != LBM_OK) return rc;
  e = cudaEventRecord(c->diag_filled[b], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_diag order");
  // final sums and the copy out on the diagnostic stream, beside later steps
  e = cudaStreamWaitEvent(c->diag_stream, c->diag_filled[b], 0);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_diag order");
  rc = check_launch(c, lbm::launch_diag_final(c->d, c->diag_io_off, c->diag_io_q, c->diag_fpi,
                                              c->diag_part[b], c->diag_done[b], c->diag_out[b],
                                              c->diag_stream),
                    "diagnostics kernel");
  if (rc != LBM_OK) return rc;
  const int k = (int)c->iolets.size();
  e = cudaMemcpyAsync(out, c->diag_out[b], (1 + k) * sizeof(double), cudaMemcpyDeviceToHost,
                      c->diag_stream);
  if (e == cudaSuccess) e = cudaEventRecord(c->diag_free[b], c->diag_stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_step_diag copy");
  c->diag_used[b] = true;
  ++c->diag_seq;
  return LBM_OK;
}

int lbm_tune(lbm_ctx* c, int32_t knob, int64_t value) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  c->gexec_steps = 0;  // a captured step graph holds the old settings: capture again
  switch (knob) {
    case LBM_TUNE_GRAPH_STEPS:
      if (value < 0 || (value & 1)) return fail(c, LBM_EINVAL, "graph steps must be even and >= 0");
      c->graph_steps = value;
      return LBM_OK;
    case LBM_TUNE_PREFETCH:
      if (value < 0) return fail(c, LBM_EINVAL, "prefetch distance must be >= 0");
      c->prefetch = value;
      return LBM_OK;
    case LBM_TUNE_BULK_SITES:
      if (value < 1 || value > 5) return fail(c, LBM_EINVAL, "bulk sites mode must be 1 to 5");
      if (value == 5 && lbm::storage_bytes(c->storage) == 2 && !c->tmap_ready) {
        int rc = make_tmap(c);
        if (rc != LBM_OK) return rc;
      }
      c->bulk_sites = (int32_t)value;
      return LBM_OK;
    case LBM_TUNE_BULK_WARPS:
      if (value != 4 && value != 8) return fail(c, LBM_EINVAL, "bulk warps per CTA must be 4 or 8");
      c->bulk_warps = (int32_t)value;
      return LBM_OK;
  }
  return fail(c, LBM_EINVAL, "unknown tuning knob for a lattice");
}

int lbm_sync(lbm_ctx* c) {
  if (!c) return LBM_EINVAL;
  int rc = sync(c, "lbm_sync");
  if (rc != LBM_OK) return rc;
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, c->d.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_sync flag");
  if (flag) {
    cudaMemsetAsync(c->d.err, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    if (flag & lbm::kErrTimeout)
      return fail(c, LBM_ETIMEOUT, "a bounded device wait gave up");
    if (flag & lbm::kErrCheck)
      return fail(c, LBM_ECHECK, "checked build: index out of range or a slot not written once");
    return fail(c, LBM_EUNSTABLE, "non-finite or non-positive density");
  }
  return LBM_OK;
}

int lbm_moments(lbm_ctx* c, double* rho, double* u, int32_t dst_is_device) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  const size_t n = (size_t)c->L.n;
  if (dst_is_device) {
    return check_launch(c, lbm::launch_moments(c->storage, c->d, odd_layout(c), rho, u, c->stream),
                        "moments kernel");
  }
  Temp tr(c, rho ? n * sizeof(double) : 0), tu(c, u ? 3 * n * sizeof(double) : 0);
  if ((rho && !tr.p) || (u && !tu.p)) return fail(c, LBM_ENOMEM, "lbm_moments: allocation");
  int rc = check_launch(c, lbm::launch_moments(c->storage, c->d, odd_layout(c),
                                               rho ? (double*)tr.p : nullptr,
                                               u ? (double*)tu.p : nullptr, c->stream),
                        "moments kernel");
  if (rc != LBM_OK) return rc;
  cudaError_t e = cudaSuccess;
  if (rho && n) e = cudaMemcpyAsync(rho, tr.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (u && n && e == cudaSuccess)
    e = cudaMemcpyAsync(u, tu.p, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_moments copy");
  return sync(c, "lbm_moments");
}

int lbm_plan_lattice(const uint8_t* labels, int32_t nx, int32_t ny, int32_t nz,
                     const lbm_iolet* iolets, int32_t n_iolets, double tau, int64_t out[8]) {
  g_build_err.clear();
  if (!out) return LBM_EINVAL;
  HostLattice L;
  std::string err;
  int rc;
  try {
    rc = lbm::build_lattice(labels, nx, ny, nz, iolets, n_iolets, tau, L, err);
  } catch (const std::bad_alloc&) {
    rc = LBM_ENOMEM;
    err = "host allocation failed";
  }
  if (rc != LBM_OK) {
    g_build_err = err;
    return rc;
  }
  out[0] = L.n;
  out[1] = (int64_t)L.wall_sites.size();
  out[2] = L.n_wall_links;
  out[3] = L.n_tiles;
  out[4] = L.n_bulk;
  out[5] = L.n_uniform;
  out[6] = L.n_irregular;
  out[7] = L.bulk_sites;
  return LBM_OK;
}

int lbm_info(const lbm_ctx* c, int64_t out[12]) {
  if (!c || !out) return LBM_EINVAL;
  const HostLattice& L = c->L;
  out[0] = L.n;
  out[1] = (int64_t)L.wall_sites.size();
  out[2] = L.n_wall_links;
  out[3] = L.n_tiles;
  out[4] = L.n_bulk;
  out[5] = L.n_uniform;
  out[6] = L.n_irregular;
  out[7] = c->step;
  out[8] = c->storage;
  out[9] = (int64_t)c->iolets.size();
  out[10] = (int64_t)c->dev_bytes;
  out[11] = L.bulk_sites;
  return LBM_OK;
}

int lbm_export_lattice(const lbm_ctx* c, int32_t* coords, int32_t* nbr, int64_t* wall_sites,
                       int64_t* wall_links) {
  if (!c) return LBM_EINVAL;
  const HostLattice& L = c->L;
  if (coords) std::memcpy(coords, L.coords.data(), L.coords.size() * sizeof(int32_t));
  if (nbr) std::memcpy(nbr, L.nbr.data(), L.nbr.size() * sizeof(int32_t));
  if (wall_sites)
    std::memcpy(wall_sites, L.wall_sites.data(), L.wall_sites.size() * sizeof(int64_t));
  if (wall_links) {
    int64_t k = 0;
    for (int64_t s = 0; s < L.n; ++s)
      for (int i = 1; i < lbm::kQ; ++i)
        if (L.nbr[(size_t)18 * s + (i - 1)] == -1) {
          wall_links[2 * k] = s;
          wall_links[2 * k + 1] = i;
          ++k;
        }
  }
  return LBM_OK;
}

int lbm_wall_state(lbm_ctx* c, double* dE, double* Uw) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  const size_t S = (size_t)c->L.n_slots;
  std::vector<double> hdE(S), hUw(3 * S);
  cudaError_t e = cudaSuccess;
  if (S) {
    e = cudaMemcpyAsync(hdE.data(), c->d.slot_dE, S * sizeof(double), cudaMemcpyDeviceToHost,
                        c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(hUw.data(), c->d.slot_Uw, 3 * S * sizeof(double),
                          cudaMemcpyDeviceToHost, c->stream);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_wall_state copy");
  int rc = sync(c, "lbm_wall_state");
  if (rc != LBM_OK) return rc;
  for (size_t w = 0; w < c->L.wall_sites.size(); ++w) {
    const int64_t m = c->L.wall_slot[w];
    if (dE) dE[w] = hdE[m];
    if (Uw)
      for (int a = 0; a < 3; ++a) Uw[3 * w + a] = hUw[(size_t)a * S + m];
  }
  return LBM_OK;
}

int lbm_reduce(lbm_ctx* c, double* out) {
  if (!c || !out) return LBM_EINVAL;
  c->err.clear();
  const int k = (int)c->iolets.size();
  int rc = check_launch(c, lbm::launch_reduce(c->storage, c->d, odd_layout(c), c->iolet_off,
                                              c->iolet_sites, c->partial, lbm::reduce_partials(),
                                              c->red_out, c->stream),
                        "reduce kernels");
  if (rc != LBM_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(out, c->red_out, (1 + k) * sizeof(double),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_reduce copy");
  return sync(c, "lbm_reduce");
}

int lbm_get_populations(lbm_ctx* c, double* f, int32_t dst_is_device) {
  if (!c || !f) return LBM_EINVAL;
  c->err.clear();
  const size_t cnt = (size_t)c->L.n * lbm::kQ;
  if (dst_is_device)
    return check_launch(c, lbm::launch_gather(c->storage, c->d, odd_layout(c), f, c->stream),
                        "gather kernel");
  Temp t(c, cnt * sizeof(double));
  if (!t.p) return fail(c, LBM_ENOMEM, "lbm_get_populations: allocation");
  int rc = check_launch(c, lbm::launch_gather(c->storage, c->d, odd_layout(c), (double*)t.p,
                                              c->stream),
                        "gather kernel");
  if (rc != LBM_OK) return rc;
  if (cnt) {
    cudaError_t e = cudaMemcpyAsync(f, t.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_get_populations copy");
  }
  return sync(c, "lbm_get_populations");
}

int lbm_set_populations(lbm_ctx* c, const double* f, int64_t step, int32_t src_is_device) {
  if (!c || !f) return LBM_EINVAL;
  if (step < 0) return fail(c, LBM_EINVAL, "step must be >= 0");
  c->err.clear();
  const size_t cnt = (size_t)c->L.n * lbm::kQ;
  const int odd = (int)(step & 1);
  if (src_is_device) {
    int rc = check_launch(c, lbm::launch_scatter(c->storage, c->d, odd, f, c->stream),
                          "scatter kernel");
    if (rc == LBM_OK) c->step = step;
    return rc;
  }
  Temp t(c, cnt * sizeof(double));
  if (!t.p) return fail(c, LBM_ENOMEM, "lbm_set_populations: allocation");
  cudaError_t e = h2d(c, (double*)t.p, f, cnt);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_set_populations copy");
  int rc = check_launch(c, lbm::launch_scatter(c->storage, c->d, odd, (double*)t.p, c->stream),
                        "scatter kernel");
  if (rc == LBM_OK) rc = sync(c, "lbm_set_populations");
  if (rc == LBM_OK) c->step = step;
  return rc;
}

size_t lbm_checkpoint_bytes(const lbm_ctx* c) {
  if (!c) return 0;
  return 4 * sizeof(uint64_t) + (size_t)lbm::kQ * c->d.npad * lbm::storage_bytes(c->storage);
}

int lbm_checkpoint_save(lbm_ctx* c, void* buf, size_t bytes) {
  if (!c || !buf) return LBM_EINVAL;
  if (bytes < lbm_checkpoint_bytes(c)) return fail(c, LBM_EINVAL, "checkpoint buffer too small");
  uint64_t* h = static_cast<uint64_t*>(buf);
  h[0] = kCkptMagic;
  h[1] = (uint64_t)c->storage | ((uint64_t)c->L.n << 8);
  h[2] = (uint64_t)c->d.npad;
  h[3] = (uint64_t)c->step;
  const size_t pb = lbm_checkpoint_bytes(c) - 4 * sizeof(uint64_t);
  cudaError_t e = cudaMemcpyAsync(h + 4, c->d.pop, pb, cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_checkpoint_save");
  return sync(c, "lbm_checkpoint_save");
}

int lbm_checkpoint_load(lbm_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return LBM_EINVAL;
  if (bytes < lbm_checkpoint_bytes(c)) return fail(c, LBM_EINVAL, "checkpoint buffer too small");
  const uint64_t* h = static_cast<const uint64_t*>(buf);
  if (h[0] != kCkptMagic || h[1] != ((uint64_t)c->storage | ((uint64_t)c->L.n << 8)) ||
      h[2] != (uint64_t)c->d.npad)
    return fail(c, LBM_EINVAL, "checkpoint does not match this lattice");
  const size_t pb = lbm_checkpoint_bytes(c) - 4 * sizeof(uint64_t);
  cudaError_t e = cudaMemcpyAsync(c->d.pop, h + 4, pb, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_checkpoint_load");
  int rc = sync(c, "lbm_checkpoint_load");
  if (rc == LBM_OK) c->step = (int64_t)h[3];
  return rc;
}

int lbm_wss(lbm_ctx* c, const int64_t* sites, const double* normals, int64_t m, double* out) {
  if (!c || m < 0 || (m > 0 && (!sites || !normals || !out))) return LBM_EINVAL;
  c->err.clear();
  if (m == 0) return LBM_OK;
  for (int64_t q = 0; q < m; ++q)
    if (sites[q] < 0 || sites[q] >= c->L.n) return fail(c, LBM_EINVAL, "site id out of range");
  Temp ts(c, m * sizeof(int64_t)), tn(c, 3 * m * sizeof(double)), to(c, m * sizeof(double));
  if (!ts.p || !tn.p || !to.p) return fail(c, LBM_ENOMEM, "lbm_wss: allocation");
  cudaError_t e = h2d(c, (int64_t*)ts.p, sites, m);
  if (e == cudaSuccess) e = h2d(c, (double*)tn.p, normals, 3 * m);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_wss copy");
  int rc = check_launch(c, lbm::launch_wss(c->storage, c->d, odd_layout(c), c->tau,
                                           (const int64_t*)ts.p, (const double*)tn.p, m,
                                           (double*)to.p, c->stream),
                        "wss kernel");
  if (rc != LBM_OK) return rc;
  e = cudaMemcpyAsync(out, to.p, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_wss copy back");
  return sync(c, "lbm_wss");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// lbm_reduce_noalloc: the FP64 diagnostics of lbm_reduce for callers that must
// not allocate device memory while the call runs - for example a monitoring
// hook that runs while another component's memory pool holds the whole device
// (a cudaMalloc there can fail or force the pool to release memory), or a
// latency-bound loop that cannot afford the device-wide synchronisation that
// cudaMalloc/cudaFree may imply.  Its scratch (per-block partial sums and the
// result) lives in the fixed device array below instead of the context's
// buffers; the call allocates nothing.
namespace {

constexpr int kNoAllocPartials = 1024;  // partial sums of the mass reduction
constexpr int kNoAllocOutputs = 256;    // 1 + n_iolets at most
// Held by every GPU that loads this library until the process exits
// (10 KiB).  Shared by every call: calls that overlap on the GPU race.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials + kNoAllocOutputs];

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
// Cached address per device, valid for the CUDA context it was looked up in:
// a device reset (or any destruction of the primary context) loads the module
// again, possibly at another address, and gives the new context a new id.
struct NoAllocSlot {
  unsigned long long ctx_id;
  double* ptr;
};
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (driver entry points
// resolved through the runtime, so the library does not link libcuda), or 0
// when it cannot be had - then the address is looked up on every call.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {  // under g_noalloc_mu
    resolved = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  }
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device and context (with that device current) and cached.
int noalloc_scratch(lbm_ctx* c, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_reduce_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(c, LBM_EINVAL, "lbm_reduce_noalloc: device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  const unsigned long long ctx = current_context_id();
  NoAllocSlot& slot = g_noalloc_slot[dev];
  if (!slot.ptr || ctx == 0 || slot.ctx_id != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(c, e, "lbm_reduce_noalloc: cudaGetSymbolAddress");
    slot.ptr = static_cast<double*>(p);
    slot.ctx_id = ctx;
  }
  *out = slot.ptr;
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_noalloc(lbm_ctx* c, double* out, int32_t out_is_device) {
  if (!c || !out) return LBM_EINVAL;
  c->err.clear();
  const int k = (int)c->iolets.size();
  if (1 + k > kNoAllocOutputs)
    return fail(c, LBM_EINVAL, "lbm_reduce_noalloc: more than 255 iolets");
  if (lbm::reduce_partials() > kNoAllocPartials)
    return fail(c, LBM_EINVAL, "lbm_reduce_noalloc: scratch smaller than the reduction grid");
  double* scratch = nullptr;
  int rc = noalloc_scratch(c, &scratch);
  if (rc != LBM_OK) return rc;
  // Every partial and every output is written by the kernels before it is
  // read, so nothing left by an earlier call needs clearing.
  double* dst = out_is_device ? out : scratch + kNoAllocPartials;
  rc = check_launch(c, lbm::launch_reduce(c->storage, c->d, odd_layout(c), c->iolet_off,
                                          c->iolet_sites, scratch, kNoAllocPartials, dst,
                                          c->stream),
                    "reduce kernels");
  if (rc != LBM_OK || out_is_device) return rc;
  cudaError_t e = cudaMemcpyAsync(out, dst, (1 + k) * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_reduce_noalloc copy");
  return sync(c, "lbm_reduce_noalloc");
}

// ---------------------------------------------------------------------------
// Ensembles: many independent lattices advanced by one launch of each step
// kernel per timestep (optionally replayed from a captured CUDA graph).

struct lbm_ensemble {
  std::vector<lbm_ctx*> members;  // not owned
  int storage = LBM_F64;
  // private streams (capturable), ordered after / before the members' streams
  cudaStream_t stream = nullptr, side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, ord_ev = nullptr;
  std::vector<cudaStream_t> member_streams;  // distinct streams of the members
  std::vector<void*> owned;       // device buffers (member 0's allocator)
  lbm::MemberDev* mem_d = nullptr;
  lbm::TileRef* map_d = nullptr;  // tile maps: bulk tiles, then boundary tiles
  int64_t n_bulk = 0, n_boundary = 0;  // tiles of all members
  int64_t* step_d = nullptr;      // device step counter of captured graphs
  std::vector<int32_t> order;     // schedule: member order in the launch numbering
  int64_t prefetch = 0;           // set from the storage at creation
  int32_t bulk_sites = 1;         // bulk kernel mode, set from the storage
  int32_t bulk_warps = 4;         // warps per CTA of the bulk kernel
  int64_t graph_steps = 0;        // 0: direct launches
  int persistent = 0;             // 1: one cooperative launch per lbm_ensemble_step
  int barrier_extra = 0;          // fault injection: arrivals the grid barrier waits for in vain
  lbm::GridSync* sync_d = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t exec_steps = 0;
  int exec_parity = -1;
  lbm::EnsembleLaunch launch{};
  std::vector<lbm::MemberDev> multi_host;  // members with multi-iolet tiles (host copies)
  std::string err;
};

namespace {

int ens_fail(lbm_ensemble* e, int code, const std::string& msg) {
  if (e) e->err = msg;
  return code;
}

int ens_cuda(lbm_ensemble* e, cudaError_t r, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(r));
  return ens_fail(e, LBM_ECUDA, buf);
}

void ens_drop_graph(lbm_ensemble* e) {
  if (e->exec) cudaGraphExecDestroy(e->exec);
  e->exec = nullptr;
  e->exec_steps = 0;
  e->exec_parity = -1;
}

// Upload the member table and the prefix tables in schedule order.
// Tile maps in schedule order: for every global bulk (boundary) tile, its
// member's position in the member table and its launch position there.
int ens_maps(lbm_ensemble* e) {
  const int n = (int)e->members.size();
  std::vector<lbm::TileRef> map((size_t)(e->n_bulk + e->n_boundary));
  size_t gb = 0, gd = (size_t)e->n_bulk;
  for (int q = 0; q < n; ++q) {
    const lbm_ctx* c = e->members[e->order[q]];
    for (int64_t k = c->d.n_boundary; k < c->d.n_tiles; ++k) map[gb++] = lbm::TileRef{q, (int32_t)k};
    for (int64_t k = 0; k < c->d.n_boundary; ++k) map[gd++] = lbm::TileRef{q, (int32_t)k};
  }
  cudaError_t r = cudaMemcpyAsync(e->map_d, map.data(), map.size() * sizeof(lbm::TileRef),
                                  cudaMemcpyHostToDevice, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);  // map is a temporary
  if (r != cudaSuccess) return ens_cuda(e, r, "ensemble tile map upload");
  e->launch.bulk_map = e->map_d;
  e->launch.boundary_map = e->map_d + e->n_bulk;
  ens_drop_graph(e);
  return LBM_OK;
}

int ens_upload(lbm_ensemble* e) {
  const int n = (int)e->members.size();
  std::vector<lbm::MemberDev> tab(n);
  for (int q = 0; q < n; ++q) {
    const lbm_ctx* c = e->members[e->order[q]];
    lbm::MemberDev& md = tab[q];
    std::memset(&md, 0, sizeof md);
    md.d = c->d;
    md.d.chk = nullptr;  // store counting covers single-lattice steps only
    md.omega = 1.0 / c->tau;
    md.omega_f = (float)md.omega;
    md.rho0 = c->rho0;
    md.rho0_f = (float)c->rho0;
    md.rho0_exact = (double)md.rho0_f == c->rho0 ? 1 : 0;
    md.elastic = c->wall_model == LBM_WALL_ELASTIC_GZS ? 1 : 0;
  }
  cudaError_t r = cudaMemcpyAsync(e->mem_d, tab.data(), n * sizeof(lbm::MemberDev),
                                  cudaMemcpyHostToDevice, e->stream);
  if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);  // tab is a temporary
  if (r != cudaSuccess) return ens_cuda(e, r, "ensemble upload");
  e->multi_host.clear();
  for (const lbm::MemberDev& md : tab)
    if (md.d.n_multi > 0) e->multi_host.push_back(md);
  e->launch.multi_host = e->multi_host.data();
  e->launch.n_multi_members = (int32_t)e->multi_host.size();
  e->launch.mem = e->mem_d;
  e->launch.n_members = n;
  e->launch.n_bulk_tiles = e->n_bulk;
  e->launch.n_boundary_tiles = e->n_boundary;
  ens_drop_graph(e);
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_ensemble_last_error(const lbm_ensemble* e) {
  return e ? e->err.c_str() : "null ensemble";
}

void lbm_ensemble_destroy(lbm_ensemble* e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  if (e->side) cudaStreamSynchronize(e->side);
  ens_drop_graph(e);
  if (!e->members.empty())
    for (void* p : e->owned) dev_free_raw(e->members[0], p);
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->join) cudaEventDestroy(e->join);
  if (e->ord_ev) cudaEventDestroy(e->ord_ev);
  if (e->side) cudaStreamDestroy(e->side);
  if (e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

int lbm_ensemble_create(lbm_ctx* const* members, int32_t n, lbm_ensemble** out) {
  if (!out || !members || n <= 0) return LBM_EINVAL;
  *out = nullptr;
  for (int q = 0; q < n; ++q)
    if (!members[q] || members[q]->storage != members[0]->storage ||
        members[q]->step != members[0]->step)
      return LBM_EINVAL;
  lbm_ensemble* e = new (std::nothrow) lbm_ensemble();
  if (!e) return LBM_ENOMEM;
  e->members.assign(members, members + n);
  e->storage = members[0]->storage;
  e->prefetch = default_prefetch(e->storage);
  e->bulk_sites = default_bulk_sites(e->storage);
  for (lbm_ctx* c : e->members)
    if (std::find(e->member_streams.begin(), e->member_streams.end(), c->stream) ==
        e->member_streams.end())
      e->member_streams.push_back(c->stream);
  e->order.resize(n);
  for (int q = 0; q < n; ++q) e->order[q] = q;
  int lo = 0, hi = 0;
  cudaError_t r = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (r == cudaSuccess) r = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
  if (r == cudaSuccess) r = cudaStreamCreateWithPriority(&e->side, cudaStreamNonBlocking, hi);
  if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming);
  if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e->join, cudaEventDisableTiming);
  if (r == cudaSuccess) r = cudaEventCreateWithFlags(&e->ord_ev, cudaEventDisableTiming);
  if (r != cudaSuccess) {
    lbm_ensemble_destroy(e);
    return LBM_ECUDA;
  }
  lbm_ctx* c0 = members[0];
  auto alloc = [&](size_t bytes) {
    void* p = dev_alloc_raw(c0, bytes);
    if (p) e->owned.push_back(p);
    return p;
  };
  for (lbm_ctx* c : e->members) {
    e->n_bulk += c->d.n_tiles - c->d.n_boundary;
    e->n_boundary += c->d.n_boundary;
  }
  e->mem_d = static_cast<lbm::MemberDev*>(alloc(n * sizeof(lbm::MemberDev)));
  e->map_d = static_cast<lbm::TileRef*>(
      alloc(std::max<int64_t>(1, e->n_bulk + e->n_boundary) * sizeof(lbm::TileRef)));
  e->step_d = static_cast<int64_t*>(alloc(sizeof(int64_t)));
  e->sync_d = static_cast<lbm::GridSync*>(alloc(sizeof(lbm::GridSync)));
  if (!e->mem_d || !e->map_d || !e->step_d || !e->sync_d) {
    lbm_ensemble_destroy(e);
    return LBM_ENOMEM;
  }
  if (ens_maps(e) != LBM_OK || ens_upload(e) != LBM_OK) {
    lbm_ensemble_destroy(e);
    return LBM_ECUDA;
  }
  *out = e;
  return LBM_OK;
}

int lbm_ensemble_tune(lbm_ensemble* e, int32_t knob, int64_t value) {
  if (!e) return LBM_EINVAL;
  e->err.clear();
  switch (knob) {
    case LBM_TUNE_PREFETCH:
      if (value < 0) return ens_fail(e, LBM_EINVAL, "prefetch distance must be >= 0");
      e->prefetch = value;
      ens_drop_graph(e);
      return LBM_OK;
    case LBM_TUNE_SCHEDULE: {
      const int n = (int)e->members.size();
      for (int q = 0; q < n; ++q) e->order[q] = q;
      if (value == 1) {  // largest members first
        std::stable_sort(e->order.begin(), e->order.end(), [&](int a, int b) {
          return e->members[a]->d.n_tiles > e->members[b]->d.n_tiles;
        });
      } else if (value != 0) {
        return ens_fail(e, LBM_EINVAL, "schedule must be 0 (given order) or 1 (largest first)");
      }
      if (ens_maps(e) != LBM_OK) return LBM_ECUDA;
      return ens_upload(e);
    }
    case LBM_TUNE_GRAPH_STEPS:
      if (value < 0 || (value & 1)) return ens_fail(e, LBM_EINVAL, "graph steps must be even");
      e->graph_steps = value;
      ens_drop_graph(e);
      return LBM_OK;
    case LBM_TUNE_PERSISTENT:
      if (value != 0 && value != 1) return ens_fail(e, LBM_EINVAL, "persistent must be 0 or 1");
      e->persistent = (int)value;
      return LBM_OK;
    case LBM_TUNE_BARRIER_EXTRA:
      if (value < 0 || value > 1024) return ens_fail(e, LBM_EINVAL, "barrier extra out of range");
      e->barrier_extra = (int)value;
      return LBM_OK;
    case LBM_TUNE_BULK_SITES:
      if (value < 1 || value > 4) return ens_fail(e, LBM_EINVAL, "bulk sites mode must be 1 to 4");
      e->bulk_sites = (int32_t)value;
      ens_drop_graph(e);
      return LBM_OK;
    case LBM_TUNE_BULK_WARPS:
      if (value != 4 && value != 8) return ens_fail(e, LBM_EINVAL, "bulk warps must be 4 or 8");
      e->bulk_warps = (int32_t)value;
      ens_drop_graph(e);
      return LBM_OK;
  }
  return ens_fail(e, LBM_EINVAL, "unknown tuning knob");
}

int lbm_ensemble_step(lbm_ensemble* e, int64_t n_steps) {
  if (!e || n_steps < 0) return LBM_EINVAL;
  e->err.clear();
  const int64_t step0 = e->members[0]->step;
  for (lbm_ctx* c : e->members)
    if (c->step != step0) return ens_fail(e, LBM_ESTATE, "members are at different steps");
  int rc = ens_upload(e);  // wall models or rho0 may have changed since the last call
  if (rc != LBM_OK) return rc;
  // start after the members' pending work
  for (cudaStream_t ms : e->member_streams) {
    cudaError_t r = cudaEventRecord(e->ord_ev, ms);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(e->stream, e->ord_ev, 0);
    if (r != cudaSuccess) return ens_cuda(e, r, "ensemble ordering");
  }
  const lbm::StepStreams ss{e->stream, e->side, e->fork, e->join};
  lbm::StepParams p{};
  p.prefetch = e->prefetch;
  p.bulk_sites = e->bulk_sites;
  p.bulk_warps = e->bulk_warps;
  int64_t done = 0;
  if (e->persistent && n_steps > 0) {
    p.step = step0;
    p.step_dev = nullptr;
    const int lr = lbm::launch_ensemble_persistent(e->storage, e->launch, p, n_steps, e->sync_d,
                                                   e->barrier_extra, e->stream);
    if (lr != 0) return ens_cuda(e, (cudaError_t)lr, "persistent ensemble launch");
    done = n_steps;
  }
  const int64_t G = e->persistent ? 0 : e->graph_steps;
  if (G > 0 && n_steps >= G) {
    const int parity = (int)(step0 & 1);
    if (!e->exec || e->exec_steps != G || e->exec_parity != parity) {
      ens_drop_graph(e);
      cudaGraph_t graph = nullptr;
      cudaError_t r = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
      for (int64_t s = 0; s < G && r == cudaSuccess; ++s) {
        p.step = parity + s;  // offset; the step is *step_d + offset - parity
        p.step_dev = e->step_d;
        p.write_state = s == G - 1 ? 1 : 0;
        const int lr = lbm::launch_ensemble_step(e->storage, e->launch, p, ss);
        if (lr != 0) r = (cudaError_t)lr;
      }
      if (r == cudaSuccess) r = (cudaError_t)lbm::launch_advance(e->step_d, G, e->stream);
      cudaError_t r2 = cudaStreamEndCapture(e->stream, &graph);
      if (r == cudaSuccess) r = r2;
      if (r == cudaSuccess) r = cudaGraphInstantiate(&e->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (r != cudaSuccess) {
        e->exec = nullptr;
        return ens_cuda(e, r, "ensemble graph capture");
      }
      e->exec_steps = G;
      e->exec_parity = parity;
    }
    // the captured kernels add `parity` back: store step - parity on the device
    const int64_t base = step0 - parity;
    cudaError_t r = cudaMemcpyAsync(e->step_d, &base, sizeof base, cudaMemcpyHostToDevice,
                                    e->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
    while (r == cudaSuccess && n_steps - done >= G) {
      r = cudaGraphLaunch(e->exec, e->stream);
      done += G;
    }
    if (r != cudaSuccess) return ens_cuda(e, r, "ensemble graph launch");
  }
  p.step_dev = nullptr;
  for (int64_t s = done; s < n_steps; ++s) {
    p.step = step0 + s;
    p.write_state = s == n_steps - 1 ? 1 : 0;
    const int lr = lbm::launch_ensemble_step(e->storage, e->launch, p, ss);
    if (lr != 0) return ens_cuda(e, (cudaError_t)lr, "ensemble step kernels");
  }
  for (lbm_ctx* c : e->members) c->step = step0 + n_steps;
  // the members' later work comes after the ensemble's
  cudaError_t r = cudaEventRecord(e->ord_ev, e->stream);
  for (cudaStream_t ms : e->member_streams)
    if (r == cudaSuccess) r = cudaStreamWaitEvent(ms, e->ord_ev, 0);
  if (r != cudaSuccess) return ens_cuda(e, r, "ensemble ordering");
  return LBM_OK;
}

int lbm_ensemble_sync(lbm_ensemble* e) {
  if (!e) return LBM_EINVAL;
  cudaError_t r = cudaStreamSynchronize(e->stream);
  if (r != cudaSuccess) return ens_cuda(e, r, "lbm_ensemble_sync");
  for (lbm_ctx* c : e->members) {
    const int rc = lbm_sync(c);
    if (rc != LBM_OK) return ens_fail(e, rc, c->err);
  }
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- warm start
// Learned initial fields (include/lbm_mlp.h); no counterpart in the paper.

namespace {

int warm_frame(lbm_ctx* c, const lbm_warm_frame* f, lbm_warm_frame* out) {
  if (!f) return fail(c, LBM_EINVAL, "warm start: NULL frame");
  const double a = std::sqrt(f->axis[0] * f->axis[0] + f->axis[1] * f->axis[1] +
                             f->axis[2] * f->axis[2]);
  if (!(a > 0.0) || !(f->length > 0.0) || !(f->radius > 0.0) || f->n_global < 0 ||
      f->n_global > LBM_WARM_MAX_GLOBAL || !(f->rho_scale != 0.0) || !(f->u_scale != 0.0) ||
      !std::isfinite(f->rho_scale) || !std::isfinite(f->u_scale))
    return fail(c, LBM_EINVAL, "warm start: invalid frame");
  *out = *f;
  for (int k = 0; k < 3; ++k) out->axis[k] = f->axis[k] / a;
  return LBM_OK;
}

int warm_coords(lbm_ctx* c) {
  if (c->coords_dev) return LBM_OK;
  int32_t* p = dev_alloc<int32_t>(c, c->L.coords.size());
  if (!p) return fail(c, LBM_ENOMEM, "warm start: coordinate allocation");
  cudaError_t e = h2d(c, p, c->L.coords.data(), c->L.coords.size());
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "warm start: coordinate copy");
  c->coords_dev = p;
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_warm_features(lbm_ctx* c, const lbm_warm_frame* frame, float* x, float* t) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  lbm_warm_frame f;
  int rc = warm_frame(c, frame, &f);
  if (rc != LBM_OK) return rc;
  if (!x) return fail(c, LBM_EINVAL, "lbm_warm_features: NULL x");
  if ((rc = warm_coords(c)) != LBM_OK) return rc;
  const size_t n = (size_t)c->L.n;
  Temp tr(c, t ? n * sizeof(double) : 0), tu(c, t ? 3 * n * sizeof(double) : 0);
  if (t && (!tr.p || !tu.p)) return fail(c, LBM_ENOMEM, "lbm_warm_features: allocation");
  if (t) {
    rc = check_launch(c, lbm::launch_moments(c->storage, c->d, odd_layout(c), (double*)tr.p,
                                             (double*)tu.p, c->stream),
                      "moments kernel");
    if (rc != LBM_OK) return rc;
  }
  rc = check_launch(c, lbm::launch_warm_features(c->coords_dev, (int64_t)n, f, (double*)tr.p,
                                                 (double*)tu.p, x, t, c->stream),
                    "warm feature kernel");
  if (rc == LBM_OK) rc = sync(c, "lbm_warm_features");
  return rc;
}

int lbm_warm_start(lbm_ctx* c, lbm_mlp* net, const lbm_warm_frame* frame) {
  if (!c) return LBM_EINVAL;
  c->err.clear();
  if (!net) return fail(c, LBM_EINVAL, "lbm_warm_start: NULL network");
  lbm_warm_frame f;
  int rc = warm_frame(c, frame, &f);
  if (rc != LBM_OK) return rc;
  int n_in = 0, n_out = 0;
  void* ns = nullptr;
  lbm::mlp_shape(net, &n_in, &n_out, &ns);
  if (n_in != f.n_global + 2 || n_out != 3)
    return fail(c, LBM_EINVAL, "lbm_warm_start: network needs n_in = n_global + 2, n_out = 3");
  if ((rc = warm_coords(c)) != LBM_OK) return rc;
  // The network's buffers are used on this context's stream: let its own
  // queued work finish first.
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(ns));
  if (e != cudaSuccess) return cuda_fail(c, e, "lbm_warm_start: network stream");
  const size_t n = (size_t)c->L.n;
  Temp tx(c, n * n_in * sizeof(float)), ty(c, n * 3 * sizeof(float));
  Temp tr(c, n * sizeof(double)), tu(c, 3 * n * sizeof(double));
  if (!tx.p || !ty.p || !tr.p || !tu.p) return fail(c, LBM_ENOMEM, "lbm_warm_start: allocation");
  rc = check_launch(c, lbm::launch_warm_features(c->coords_dev, (int64_t)n, f, nullptr, nullptr,
                                                 (float*)tx.p, nullptr, c->stream),
                    "warm feature kernel");
  if (rc == LBM_OK)
    rc = check_launch(c, lbm::mlp_forward_on(net, (const float*)tx.p, (int64_t)n, (float*)ty.p,
                                             c->stream),
                      "network forward");
  if (rc == LBM_OK)
    rc = check_launch(c, lbm::launch_warm_fields(c->coords_dev, (int64_t)n, f,
                                                 (const float*)ty.p, (double*)tr.p,
                                                 (double*)tu.p, c->stream),
                      "warm field kernel");
  if (rc == LBM_OK)
    rc = check_launch(c, lbm::launch_init(c->storage, c->d, (double*)tr.p, (double*)tu.p,
                                          c->stream),
                      "init kernel");
  const int rs = sync(c, "lbm_warm_start");
  if (rc == LBM_OK) rc = rs;
  if (rc == LBM_OK) c->step = 0;
  return rc;
}

}  // extern "C"
