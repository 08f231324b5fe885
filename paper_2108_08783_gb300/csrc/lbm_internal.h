// Internal declarations of the GB300 elastic-wall D3Q19 library: the host
// lattice (built once from voxel labels) and the device-side views the
// kernels use.  Not part of the public C ABI (see include/lbm.h).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "../../include/lbm_mlp.h"

namespace lbm {

constexpr int kQ = 19;
constexpr int kTile = 32;          // sites per tile = one warp

// Flag bits shared by TileDesc::mask and the per-slot masks.  Bits 1..18 mark
// the non-fluid directions (wall or iolet links).
constexpr uint32_t kDirBits = 0x7FFFEu;
constexpr uint32_t kMultiIolet = 1u << 19; // site links into two or more iolets: the
                                           // per-link codes of the neighbour table decide
constexpr uint32_t kValid = 1u << 28;      // slot holds a site (slot masks only)
// Iolet-link words (slot_io): bits 1..18 = the non-fluid link is an iolet link;
// bits 20..31 = the site's iolet id (its velocity inlet if it has one).
constexpr int kIoletShift = 20;
constexpr uint32_t kIoletIdBits = 0xFFFu << kIoletShift;
constexpr int kMaxIolets = 4095;
constexpr uint32_t kHasInlet = 1u << 29;   // a velocity-inlet link is present
constexpr uint32_t kHasWall = 1u << 30;    // a wall link is present
constexpr uint32_t kIrregular = 1u << 31;  // tile: fluid-link offsets differ between lanes
// Irregular tile whose lanes fall into at most kMaxSegments runs of consecutive
// lanes that each share one offset per direction (tile masks only); its
// segment table replaces the per-site neighbour rows on odd steps.
constexpr uint32_t kSegmented = 1u << 20;
constexpr int kMaxSegments = 4;
// Segment table of a boundary tile, in 32-bit words: [0..3] first lane of
// each segment (32 for an unused one), then [4 + 18 q + (i - 1)] the offset
// nbr(x, i) - x of segment q's fluid links in direction i; padded to 80.
constexpr int kSegWords = 80;

// Sticky device error bits (ctx->err).
constexpr int kErrUnstable = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrCheck = 4;  // checked builds: index out of range / slot not written once

// One tile of 32 consecutive sites, 80 bytes, read by one warp (lanes 0..19).
//  bulk tile: mask == 0 and code[i-1] = nbr(x, i) - x, the same for every
//    lane; slot = -1.
//  coherent boundary tile: some links leave the fluid (per-site masks in the
//    slot arrays), and in every direction the lanes whose link is fluid share
//    one offset code[i-1]; mask carries kHasWall / kHasInlet and the union of
//    the non-fluid directions; slot = first slot.
//  irregular tile (kIrregular): fluid-link offsets differ between lanes; the
//    per-site neighbour table in the slot arrays gives every link.
struct alignas(16) TileDesc {
  int32_t code[18];
  uint32_t mask;
  int32_t slot;
};
static_assert(sizeof(TileDesc) == 80, "TileDesc must be 80 bytes");

// The same descriptor in launch order (boundary tiles first, then bulk tiles):
// `tile` replaces `slot`; a boundary tile at launch position k owns slots
// [32 k, 32 k + 32).
struct alignas(16) LaunchDesc {
  int32_t code[18];
  uint32_t mask;
  int32_t tile;
};
static_assert(sizeof(LaunchDesc) == 80, "LaunchDesc must be 80 bytes");

// Iolet as the kernels see it.
struct IoletDev {
  int32_t kind;   // LBM_IOLET_VELOCITY / LBM_IOLET_DENSITY
  int32_t steady; // 1: no oscillating term (period <= 0)
  double rho;
  double u_mean, u_amp, period, phase;
  double axis[3];  // unit vector
  double pad;
  // The same constants for the FP32 compute paths, rounded once on the host:
  // the phase th = 2 pi n / T + phase as a 64-bit fixed-point fraction of a
  // period, frac(n / T + phase / 2 pi) = (phase_off + n phase_inc) / 2^64
  // (mod 1; integer arithmetic, no FP64 in the step kernels), and float
  // copies of rho, rho - 1, u_mean, u_amp and the axis.
  uint64_t phase_inc;
  uint64_t phase_off;
  float rho_f, drho_f, u_mean_f, u_amp_f;
  float axis_f[3];
  float pad_f;
};
static_assert(sizeof(IoletDev) % 16 == 0, "IoletDev alignment");

// 2^64 x as an integer, for a fraction x in [0, 1) (anything else gives 0).
inline uint64_t frac_to_u64(double x) {
  if (!(x >= 0.0) || x >= 1.0) return 0;
  return (uint64_t)std::ldexp(x, 64);
}

// Allocator whose resize() leaves new elements uninitialised, for the large
// host arrays that the builder's threads write in full (first touch happens
// in parallel, not in a serial zero fill).
template <class T>
struct NoInitAlloc : std::allocator<T> {
  using value_type = T;
  NoInitAlloc() = default;
  template <class U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <class U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using big_vector = std::vector<T, NoInitAlloc<T>>;

// Host-side lattice produced by build_lattice().
struct HostLattice {
  int32_t nx = 0, ny = 0, nz = 0;
  int64_t n = 0;                  // fluid sites
  big_vector<int32_t> coords;     // [n][3]
  big_vector<int32_t> nbr;        // [n][18]
  std::vector<int64_t> wall_sites;
  int64_t n_wall_links = 0;
  // tiles (32 sites each, in site order)
  int64_t n_tiles = 0;
  std::vector<TileDesc> tiles;
  std::vector<LaunchDesc> launch;   // boundary tiles (ascending), then bulk tiles
  int64_t n_bulk = 0, n_uniform = 0, n_irregular = 0, bulk_sites = 0;  // uniform = coherent
  // boundary slots (32 per boundary tile, in tile order)
  int64_t n_slots = 0;
  std::vector<uint32_t> slot_mask;   // [n_slots]
  std::vector<uint32_t> slot_io;     // [n_slots] iolet-link word (see kIoletShift)
  big_vector<int32_t> slot_nbr;      // [18][n_slots] absolute neighbour or non-fluid code
  std::vector<double> slot_prof;     // [3][n_slots] inlet shape p0, ps, pc
  std::vector<int64_t> wall_slot;    // [n_wall_sites] slot of each wall site
  std::vector<int32_t> seg_tab;      // [n_boundary tiles][kSegWords] segment tables
  std::vector<int32_t> multi_tiles;  // launch positions of boundary tiles with a site
                                     // linked to two or more iolets
  // iolet site lists (sites with a link into iolet k), CSR
  std::vector<int64_t> iolet_off;    // [n_iolets + 1]
  std::vector<int64_t> iolet_sites;
};

// Builds the lattice; returns LBM_OK or LBM_EINVAL with a message.
int build_lattice(const uint8_t* labels, int32_t nx, int32_t ny, int32_t nz,
                  const lbm_iolet* iolets, int32_t n_iolets, double tau, HostLattice& out,
                  std::string& err);

// Device views --------------------------------------------------------------

struct DevLattice {
  void* pop = nullptr;   // [19][npad] storage elements
  int64_t npad = 0;
  int64_t n = 0;
  const TileDesc* tiles = nullptr;
  const LaunchDesc* launch = nullptr;  // boundary tiles (ascending), then bulk tiles
  int64_t n_tiles = 0;
  const uint32_t* slot_mask = nullptr;
  const uint32_t* slot_io = nullptr;
  const int32_t* slot_nbr = nullptr;   // [18][slot_stride]
  // per-slot inlet profile [3][slot_stride] (p0, ps, pc) and wall F, in the
  // compute type (double for F64 storage, float otherwise)
  const void* slot_prof = nullptr;
  const void* slot_F = nullptr;
  const double* slot_kappa = nullptr;  // kappa c_s^2 = kappa / 3 (per slot), FP64 (tube law)
  double* slot_dE = nullptr;
  double* slot_Uw = nullptr;           // [3][slot_stride]
  int64_t slot_stride = 0;
  const IoletDev* iolets = nullptr;
  int32_t n_iolets = 0;
  int* err = nullptr;
  int64_t n_boundary = 0;  // boundary tiles = leading entries of the launch order
  int* chk = nullptr;      // checked builds: stores per population slot this step, [19][npad]
  const int32_t* seg_tab = nullptr;      // [n_boundary][kSegWords] (segmented irregular tiles)
  const int32_t* multi_tiles = nullptr;  // boundary tiles with multi-iolet sites
  int64_t n_multi = 0;
  // fused diagnostics (steps with StepParams::diag): per launch position the
  // tile's sum of rho - 1 over its sites; the momentum rho u of every lane of
  // the boundary tiles that have sites with iolet links, [3][diag_jstride],
  // the tile at boundary position k at lanes 32 diag_iotile[k] + (0..31)
  double* diag_mass = nullptr;
  double* diag_j = nullptr;
  const int32_t* diag_iotile = nullptr;  // [n_boundary], -1: no iolet links
  int64_t diag_jstride = 0;
};

struct StepParams {
  double omega;      // 1 / tau
  float omega_f;     // (float) omega, for the FP32 compute paths
  int32_t pad0;
  double rho0;
  float rho0_f;        // (float) rho0
  int32_t rho0_exact;  // rho0 == (double) rho0_f
  int32_t elastic;   // 1: elastic GZS wall, 0: bounce-back
  int32_t write_state;
  int64_t step;      // step index (plus *step_dev when step_dev is set)
  int64_t prefetch;  // L2 prefetch distance in tiles of launch order (0: off)
  const int64_t* step_dev;  // device step counter (captured graphs), or NULL
  int32_t bulk_sites;       // bulk kernel mode (LBM_TUNE_BULK_SITES)
  int32_t bulk_warps;       // warps per CTA of the bulk kernel: 4 or 8
  int32_t diag;             // 1: the step kernels also write the fused diagnostics
  int32_t n_sms;            // SMs of the device (fixed-grid kernels)
  const void* tmap;         // host CUtensorMap of the populations (staged rows), or NULL
};

// One member of an ensemble: its device view and its wall constants.
struct MemberDev {
  DevLattice d;
  double omega;
  double rho0;
  int32_t elastic;
  float omega_f;  // (float) omega
  float rho0_f;   // (float) rho0
  int32_t rho0_exact;
};



// Kernel launchers (kernels.cu); storage is LBM_F64 ... LBM_BF16S.
// All return cudaError_t values cast to int.
// Streams and events of one step: the boundary kernel runs on `side`,
// forked from and joined back into `main` with the two events.
struct StepStreams {
  void* main;
  void* side;
  void* fork;
  void* join;
};
// events: NULL, or three cudaEvent_t recorded on the main stream before the
// fork, after the bulk kernel and after the join.
int launch_step(int storage, const DevLattice& d, const StepParams& p, const StepStreams& ss,
                void* const* events);

// A tile of an ensemble: its member and its launch position in that member.
struct TileRef {
  int32_t member;
  int32_t k;
};

// Ensemble launch: the members' bulk (boundary) tiles are numbered in
// schedule order; bulk_map[g] (boundary_map[g]) names the member and launch
// position of global bulk (boundary) tile g.
struct EnsembleLaunch {
  const MemberDev* mem;
  const TileRef* bulk_map;      // [n_bulk_tiles]
  const TileRef* boundary_map;  // [n_boundary_tiles]
  int32_t n_members;
  int64_t n_bulk_tiles, n_boundary_tiles;
  const MemberDev* multi_host;  // host copies of the members with multi-iolet tiles
  int32_t n_multi_members;
};
int launch_ensemble_step(int storage, const EnsembleLaunch& e, const StepParams& p,
                         const StepStreams& ss);

// Persistent ensemble kernel: one cooperative launch advances every member by
// n_steps, CTAs taking chunks of tiles from a device counter and meeting at a
// grid barrier after each step (bounded spin: a barrier that does not complete
// sets kErrTimeout in member 0's flag and every CTA returns).  `sync` is
// device memory the launcher clears; `extra_arrivals` > 0 makes every barrier
// wait for arrivals that never come (fault-injection hook for tests).
struct GridSync {
  unsigned int arrive;
  unsigned int gen;
  unsigned int abort;
  unsigned int pad;
  unsigned long long work[2];
};
int launch_ensemble_persistent(int storage, const EnsembleLaunch& e, const StepParams& p,
                               int64_t n_steps, GridSync* sync, int extra_arrivals,
                               void* stream);
int launch_advance(int64_t* step_dev, int64_t by, void* stream);
int launch_set_step(int64_t* step_dev, int64_t value, void* stream);
int launch_init(int storage, const DevLattice& d, const double* rho, const double* u,
                void* stream);
int launch_gather(int storage, const DevLattice& d, int odd_layout, double* f_out, void* stream);
int launch_scatter(int storage, const DevLattice& d, int odd_layout, const double* f_in,
                   void* stream);
int launch_moments(int storage, const DevLattice& d, int odd_layout, double* rho, double* u,
                   void* stream);
int launch_reduce(int storage, const DevLattice& d, int odd_layout, const int64_t* iolet_off,
                  const int64_t* iolet_sites, double* partial, int n_partial, double* out,
                  void* stream);
int launch_wss(int storage, const DevLattice& d, int odd_layout, double tau,
               const int64_t* sites, const double* normals, int64_t m, double* out,
               void* stream);
size_t storage_bytes(int storage);
// Fused diagnostics: the final sums of a step run with StepParams::diag into
// out[1 + n_iolets]; fpi = diag_flux_blocks(largest iolet site count) blocks
// per iolet, part: diag_blocks(n_iolets, fpi) doubles, done: a zeroed counter.
int launch_diag_final(const DevLattice& d, const int64_t* io_off, const int64_t* io_q, int fpi,
                      double* part, unsigned* done, double* out, void* stream);
int diag_blocks(int n_iolets, int fpi);
int diag_flux_blocks(int64_t max_sites);
// Checked builds: flag every population slot not stored exactly once since the
// last call (padding slots: never), then clear the counts.
int launch_check_counts(const DevLattice& d, void* stream);

// Learned warm start (mlp.cu): the network's forward pass on a given stream
// (n rows in chunks of its batch size, using its activation buffers), its
// shape and stream, and the per-site feature / field kernels.
int mlp_forward_on(lbm_mlp* net, const float* x, int64_t n, float* y, void* stream);
void mlp_shape(const lbm_mlp* net, int* n_in, int* n_out, void** stream);
int launch_warm_features(const int32_t* coords, int64_t n, const lbm_warm_frame& f,
                         const double* rho, const double* u, float* x, float* t, void* stream);
int launch_warm_fields(const int32_t* coords, int64_t n, const lbm_warm_frame& f, const float* y,
                       double* rho, double* u, void* stream);

int reduce_partials();

}  // namespace lbm
