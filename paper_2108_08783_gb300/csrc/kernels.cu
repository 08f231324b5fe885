// GB300 (sm_103a) kernels of the elastic-wall D3Q19 LBGK step.
//
// Layout in HBM: populations are one array per direction, pop[i][x] (structure
// of arrays, npad elements per direction), sites in canonical z-fastest order,
// streamed in place with the AA pattern:
//   even step: site x reads slot (x, i), collides and writes f*_i to (x, opp i);
//   odd step:  site x reads direction j from (x - c_j, opp j), collides and
//              writes f*_i to (x + c_i, i).
// Every slot is read and written by one site per step, so the kernels need no
// second buffer and no synchronisation between sites.  A link that leaves the
// fluid (wall, inlet or outlet) instead writes the boundary population into
// (x, opp i) on both parities, which is exactly where x reads direction opp i
// on the next step.
//
// Arithmetic (Sec. 2.1): with g_i = f_i - w_i, drho = sum g_i,
//   rho u = sum g_i c_i, g_i^eq = w_i (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)),
//   g*_i = g_i + (g_i^eq - g_i)/tau   (Eq. LBE_SRT, Eq. feq with the 1/2 factors).
// Boundary populations (Sec. 2.3, 2.4, 3), for a link i leaving the fluid at
// x, j = opp(i):
//   wall, elastic: f_j = f^eq_j(rho, U_w) + (1 - 1/tau)(f_j - f^eq_j(rho, u)),
//     U_w = (F + dr - 1)/dr u, dr = 1 + kappa max(0, (rho - rho0)/3) (FP64);
//   wall, bounce-back: f_j = f*_i;
//   velocity inlet: the GZS form with (rho, u_in(x, n));
//   density outlet: the GZS form with (rho_out, u).
//
// One kernel per step (k_step), one warp per tile of 32 sites: bulk tiles
// (all 18 links fluid) take a branch-free path with 18 neighbour offsets per
// tile; boundary tiles first stage their per-site link data (link masks, F,
// kappa, inlet profile and, on odd steps, per-site neighbours) into shared
// memory with cp.async.bulk copies completing on an mbarrier.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>
#include <utility>

#include "d3q19.h"
#include "lbm_internal.h"

namespace lbm {
namespace {

// ------------------------------------------------------------------ helpers

template <int... Is, class F>
__device__ __forceinline__ void for_seq(std::integer_sequence<int, Is...>, F&& f) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void unroll(F&& f) {
  for_seq(std::make_integer_sequence<int, N>{}, f);
}

template <class C>
__device__ __forceinline__ constexpr C weight(int i) {
  return i == 0 ? C(1.0 / 3.0) : (i <= 6 ? C(1.0 / 18.0) : C(1.0 / 36.0));
}

// c_i . u for direction I, written without multiplications by 0 or +-1.
template <int I, class C>
__device__ __forceinline__ C cdot(C ux, C uy, C uz) {
  constexpr int p = (I + 1) / 2;
  C d;
  if constexpr (p == 1) d = ux;
  else if constexpr (p == 2) d = uy;
  else if constexpr (p == 3) d = uz;
  else if constexpr (p == 4) d = ux + uy;
  else if constexpr (p == 5) d = ux - uy;
  else if constexpr (p == 6) d = ux + uz;
  else if constexpr (p == 7) d = ux - uz;
  else if constexpr (p == 8) d = uy + uz;
  else d = uy - uz;
  if constexpr (I & 1) return d;
  else return -d;
}

// Shifted equilibrium g^eq_I = f^eq_I - w_I for density 1 + drho and velocity u;
// usq = 1.5 u.u.
template <int I, class C>
__device__ __forceinline__ C geq(C drho, C rho, C ux, C uy, C uz, C usq) {
  if constexpr (I == 0) {
    return weight<C>(0) * (drho - rho * usq);
  } else {
    const C cu = cdot<I, C>(ux, uy, uz);
    return weight<C>(I) * (drho + rho * (C(3) * cu + C(4.5) * cu * cu - usq));
  }
}

// ------------------------------------------------------------- storage codecs
// Loads of 16-bit populations (one site's value, or a packed pair) with an
// L2 prefetch-size hint: the L2 fetches the aligned 256-byte block around the
// requested sectors from DRAM in one request. On the long tube this makes the
// FP16S step 2.3 % faster than plain loads (the inline loads also leave the
// paired bulk kernels fewer spills); FP32 populations measured 1 % slower with
// the same loads and keep plain ones.
__device__ __forceinline__ uint32_t ld_pop_b32(const void* p) {
  uint32_t v;
  asm volatile("ld.global.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned short ld_pop_u16(const void* p) {
  unsigned short v;
  asm volatile("ld.global.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}

// Every storage type holds g = f - w (the deviation from the rest
// equilibrium).  ld/st convert between the stored value and g in the compute
// type C; get/put convert between the stored value and f in double.
template <class S>
struct Codec;
template <>
struct Codec<double> {
  using C = double;  // compute type
  static __device__ __forceinline__ C ld(const double* p, int) { return *p; }
  static __device__ __forceinline__ void st(double* p, int, C g) { *p = g; }
  static __device__ __forceinline__ double get(const double* p, int i) { return *p + weight<double>(i); }
  static __device__ __forceinline__ void put(double* p, int i, double f) { *p = f - weight<double>(i); }
  static __device__ __forceinline__ void st_init(double* p, double g) { *p = g; }
};
template <>
struct Codec<float> {
  using C = float;
  static __device__ __forceinline__ C ld(const float* p, int) { return *p; }
  static __device__ __forceinline__ void st(float* p, int, C g) { *p = g; }
  static __device__ __forceinline__ double get(const float* p, int i) {
    return (double)*p + weight<double>(i);
  }
  static __device__ __forceinline__ void put(float* p, int i, double f) {
    *p = (float)(f - weight<double>(i));
  }
  static __device__ __forceinline__ void st_init(float* p, double g) { *p = (float)g; }
};
template <>
struct Codec<__half> {
  using C = float;
  static __device__ __forceinline__ C ld(const __half* p, int) {
    return __half2float(__ushort_as_half(ld_pop_u16(p)));
  }
  static __device__ __forceinline__ void st(__half* p, int, C g) { *p = __float2half_rn(g); }
  static __device__ __forceinline__ double get(const __half* p, int i) {
    return (double)__half2float(*p) + weight<double>(i);
  }
  static __device__ __forceinline__ void put(__half* p, int i, double f) {
    *p = __float2half_rn((float)(f - weight<double>(i)));
  }
  static __device__ __forceinline__ void st_init(__half* p, double g) { *p = __float2half_rn((float)g); }
};
template <>
struct Codec<__nv_bfloat16> {
  using C = float;
  static __device__ __forceinline__ C ld(const __nv_bfloat16* p, int) {
    return __uint_as_float((uint32_t)ld_pop_u16(p) << 16);
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, int, C g) { *p = __float2bfloat16_rn(g); }
  static __device__ __forceinline__ double get(const __nv_bfloat16* p, int i) {
    return (double)__bfloat162float(*p) + weight<double>(i);
  }
  static __device__ __forceinline__ void put(__nv_bfloat16* p, int i, double f) {
    *p = __float2bfloat16_rn((float)(f - weight<double>(i)));
  }
  static __device__ __forceinline__ void st_init(__nv_bfloat16* p, double g) { *p = __float2bfloat16_rn((float)g); }
};

// ------------------------------------------------------------------ collision

// Sum over the warp's 32 lanes in a fixed butterfly order (every lane gets it).
template <class T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip(double v) { return __drcp_rn(v); }

// Explicitly rounded multiply and fused multiply-add.  The boundary rule below
// is written once and evaluated in an unrolled and a looped form; pinning its
// operations makes both forms round identically (no compiler choice of what
// to contract).
__device__ __forceinline__ float mul_pin(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_pin(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_pin(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_pin(double a, double b, double c) { return __fma_rn(a, b, c); }

// The relaxation rate 1/tau in the compute type: the FP32 paths take the copy
// rounded on the host, so no step kernel converts from FP64 (GB300 issues one
// FP64 warp instruction in the time of dozens of FP32 ones).
template <class C>
__device__ __forceinline__ C omega_as(double w, float wf);
template <>
__device__ __forceinline__ double omega_as<double>(double w, float) { return w; }
template <>
__device__ __forceinline__ float omega_as<float>(double, float wf) { return wf; }

// Velocity inlet (Sec. 3) of a site with profile values (p0, ps, pc) at step
// n: u_in = axis (u_mean p0 + u_amp (ps sin th + pc cos th)),
// th = 2 pi n / T + phase.  FP64 paths take sin/cos of th in FP64, as the
// oracle does.  FP32 paths take th from the iolet's 64-bit fixed-point phase
// (frac(n / T + phase / 2 pi) in integer arithmetic, exact modulo one
// period), keep its top 24 bits (a phase error below 2^-24 of a period,
// ~4e-7 rad) and evaluate sinpi/cospi and the profile in FP32.
__device__ __forceinline__ void inlet_velocity(const IoletDev& io, int64_t n, double p0, double ps,
                                               double pc, double& ux, double& uy, double& uz) {
  double g = mul_pin(io.u_mean, p0);
  if (!io.steady) {
    double sn, cs;
    sincos(2.0 * M_PI * (double)n / io.period + io.phase, &sn, &cs);
    g = fma_pin(io.u_amp, fma_pin(ps, sn, mul_pin(pc, cs)), g);
  }
  ux = mul_pin(g, io.axis[0]);
  uy = mul_pin(g, io.axis[1]);
  uz = mul_pin(g, io.axis[2]);
}
__device__ __forceinline__ void inlet_velocity(const IoletDev& io, int64_t n, float p0, float ps,
                                               float pc, float& ux, float& uy, float& uz) {
  float g = mul_pin(io.u_mean_f, p0);
  if (!io.steady) {
    const uint64_t ph = io.phase_off + (uint64_t)n * io.phase_inc;  // mod 2^64
    const float t = (float)(uint32_t)(ph >> 40) * 0x1p-24f;           // [0, 1)
    float sn, cs;
    sincospif(2.0f * t, &sn, &cs);
    g = fma_pin(io.u_amp_f, fma_pin(ps, sn, mul_pin(pc, cs)), g);
  }
  ux = mul_pin(g, io.axis_f[0]);
  uy = mul_pin(g, io.axis_f[1]);
  uz = mul_pin(g, io.axis_f[2]);
}

// Tube law (Sec. 2.4): the wall expansion dE = kappa c_s^2 max(0, rho - rho0)
// in FP64, Kw = kappa c_s^2 (Sec. 2.3 pressure p - P0 = c_s^2 (rho - rho0)).
// FP64 compute: as written.  FP32 compute, with rho0 a float (p.rho0_exact)
// and rho within [rho0/2, 2 rho0]: rho - rho0 is exact in FP32 (Sterbenz), so
// the FP64 result is the same bits from one conversion and one FP64 multiply
// instead of two conversions, an FP64 add and an FP64 compare; other lanes
// take the FP64 difference.
__device__ __forceinline__ double tube_law(double Kw, double rho, const StepParams& p) {
  const double dp = rho - p.rho0;
  return Kw * (dp > 0.0 ? dp : 0.0);
}
// (the FP64 difference out of line, so that the compiler branches around it
// instead of issuing it predicated off on every lane)
__device__ __noinline__ double tube_law_fp64(double Kw, float rho, double rho0) {
  const double dp = (double)rho - rho0;
  return Kw * (dp > 0.0 ? dp : 0.0);
}
__device__ __forceinline__ double tube_law(double Kw, float rho, const StepParams& p) {
  if (p.rho0_exact && rho >= 0.5f * p.rho0_f && rho <= 2.0f * p.rho0_f)
    return Kw * (double)fmaxf(rho - p.rho0_f, 0.0f);
  return tube_law_fp64(Kw, rho, p.rho0);
}

// Density outlet state rho_out and rho_out - 1 in the compute type.
__device__ __forceinline__ void outlet_density(const IoletDev& io, double& r, double& dr) {
  r = io.rho;
  dr = io.rho - 1.0;
}
__device__ __forceinline__ void outlet_density(const IoletDev& io, float& r, float& dr) {
  r = io.rho_f;
  dr = io.drho_f;
}

template <class C>
struct Mom {
  C drho, rho, ux, uy, uz, usq;
};

// 1 / (1 + drho) to about one rounding of the exact value, from r = 1 + drho
// (rounded) and a reciprocal estimate y of r: the rounding error of r,
// d = drho - (r - 1), is exact (r - 1 is exact for r in [1/2, 2]), and one
// Newton step on the residual 1 - y (r + d) removes both d and the error of y.
// Without it the rounding of r (2^-24 relative in FP32) enters every velocity
// u = j / rho once per step.
template <class C>
__device__ __forceinline__ C inv_one_plus(C drho, C r, C y) {
  const C d = drho - (r - C(1));
  const C e = fma_pin(-y, d, fma_pin(-y, r, C(1)));
  return fma_pin(y, e, y);
}

// Eqs. (Density), (Momentum) on shifted populations (sum w_i c_i = 0).
template <class C>
__device__ __forceinline__ Mom<C> moments(const C (&g)[kQ]) {
  Mom<C> m;
  const C a1 = g[1] - g[2], a3 = g[3] - g[4], a5 = g[5] - g[6], a7 = g[7] - g[8];
  const C a9 = g[9] - g[10], a11 = g[11] - g[12], a13 = g[13] - g[14];
  const C a15 = g[15] - g[16], a17 = g[17] - g[18];
  m.drho = ((g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]))) +
           (((g[7] + g[8]) + (g[9] + g[10])) + ((g[11] + g[12]) + (g[13] + g[14]))) +
           ((g[15] + g[16]) + (g[17] + g[18]));
  const C jx = (a1 + a7) + (a9 + a11) + a13;
  const C jy = (a3 + a7) - (a9 - a15) + a17;
  const C jz = (a5 + a11) - (a13 - a15) - a17;
  m.rho = C(1) + m.drho;
  const C inv = inv_one_plus(m.drho, m.rho, recip(m.rho));
  m.ux = jx * inv;
  m.uy = jy * inv;
  m.uz = jz * inv;
  m.usq = C(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
  return m;
}

// BGK relaxation (Eq. LBE_SRT): gs_i = g_i + omega (g^eq_i - g_i).
template <class C>
__device__ __forceinline__ void relax(const C (&g)[kQ], C (&gs)[kQ], const Mom<C>& m, C omega) {
  unroll<kQ>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const C e = geq<i, C>(m.drho, m.rho, m.ux, m.uy, m.uz, m.usq);
    gs[i] = g[i] + omega * (e - g[i]);
  });
}

template <class C>
__device__ __forceinline__ bool unstable(C rho) {
  return !(rho > C(0)) || !(rho < C(1e30));
}

// --------------------------------------------------------- async bulk copies

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// Global -> shared copy of `bytes` (multiple of 16, both ends 16-byte aligned)
// completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Asynchronous prefetch of `bytes` (multiple of 16, 16-byte aligned) into L2.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(src)),
               "r"(bytes)
               : "memory");
}
// Asynchronous 8-byte global -> shared copy: no register holds the value while
// it is in flight; the copying thread waits for its own copies with
// cp_async_wait_all before reading them.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)),
               "l"(__cvta_generic_to_global(gmem))
               : "memory");
}
// one element of the compute type (4 or 8 bytes)
__device__ __forceinline__ void cp_async_elem(float* smem, const float* gmem) { cp_async4(smem, gmem); }
__device__ __forceinline__ void cp_async_elem(double* smem, const double* gmem) { cp_async8(smem, gmem); }
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: each try_wait suspends for a hardware-chosen interval, so
// the limit is reached only if the copies never complete.
constexpr uint32_t kWaitLimit = 1u << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// --------------------------------------------------------------- step kernels
//
// One warp per tile of 32 consecutive sites; the launch-ordered descriptor
// list holds the boundary tiles first and the bulk tiles after them.  Two
// kernels per step, on two streams so that they overlap (they touch disjoint
// slots):
//   k_bulk over the bulk tiles: branch-free update with the tile's 18
//     neighbour offsets, lean enough in registers to keep many warps resident,
//     and an L2 prefetch (cp.async.bulk.prefetch) of the populations of the
//     tile `prefetch` positions ahead;
//   k_boundary over the boundary tiles: every lane reads its site's link
//     masks (which links leave the fluid, which of those are iolet links, the
//     iolet id), F, kappa and inlet profile in the same round trip as the
//     tile descriptor; on odd steps of an irregular tile, lane 0 stages the
//     tile's per-site neighbour table into the warp's shared memory with
//     cp.async.bulk copies completing on the warp's mbarrier; then every lane
//     applies the collision and, for each link leaving the fluid, the
//     boundary rule.

__device__ __forceinline__ int32_t lds_volatile(const int32_t* p) {
  return *static_cast<const volatile int32_t*>(p);
}

// Checked builds (-DLBM_CHECKED): every population store of a step kernel is
// counted per slot (a separate kernel then requires exactly one per slot), and
// neighbour indices are range-checked; a violation sets kErrCheck and skips
// the access instead of trapping.
#ifdef LBM_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
template <class S>
__device__ __forceinline__ void chk_count(int* chk, const S* P0, const S* p, int64_t lim, int* err) {
  if constexpr (kChecked) {
    if (!chk) return;
    const int64_t i = p - P0;
    if (i < 0 || i >= lim) atomicOr(err, kErrCheck);
    else atomicAdd(chk + i, 1);
  }
}
__device__ __forceinline__ bool chk_site(int64_t y, int64_t n, int* err) {
  if constexpr (kChecked) {
    if (y < 0 || y >= n) {
      atomicOr(err, kErrCheck);
      return false;
    }
  }
  return true;
}

// Branch-free update of a site whose 18 links are fluid.
// Returns the site's rho - 1 (for the fused mass diagnostic).  With SLOT the
// whole warp (every lane updating a site) adds the lanes' rho - 1 as soon as
// the moments are formed and lane 0 writes the sum to *slot, so nothing of it
// stays live through the stores.
template <class S, bool ODD, bool SLOT = false>
__device__ __forceinline__ typename Codec<S>::C bulk_update(S* P, int64_t np, int64_t x,
                                                            const int32_t* dsc,
                                                            typename Codec<S>::C omega, int* err,
                                                            int* chk, double* slot = nullptr) {
  using Cd = Codec<S>;
  using C = typename Cd::C;
  C g[kQ];
  unroll<kQ>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int o = dir_opp(j);
    if constexpr (!ODD || j == 0) g[j] = Cd::ld(P + j * np + x, j);
    else g[j] = Cd::ld(P + o * np + x + dsc[o - 1], j);
  });
  const Mom<C> m = moments(g);
  if constexpr (SLOT) {
    const C sum = warp_sum(m.drho);
    if ((threadIdx.x & 31) == 0) *slot = (double)sum;
  }
  if (unstable(m.rho)) atomicOr(err, kErrUnstable);
  Cd::st(P + x, 0, g[0] + omega * (geq<0, C>(m.drho, m.rho, m.ux, m.uy, m.uz, m.usq) - g[0]));
  chk_count(chk, P, P + x, kQ * np, err);
  // Opposite directions a, b = opp(a) share c_b = -c_a, so their shifted
  // equilibria split into an even part w (drho + rho (4.5 cu^2 - 1.5 u^2)) and
  // an odd part 3 w rho cu: g^eq_a = even + odd, g^eq_b = even - odd.
  const C wd1 = m.drho * C(1.0 / 18.0), wd2 = m.drho * C(1.0 / 36.0);
  const C wr1 = m.rho * C(1.0 / 18.0), wr2 = m.rho * C(1.0 / 36.0);
  const C w3r1 = m.rho * C(3.0 / 18.0), w3r2 = m.rho * C(3.0 / 36.0);
  unroll<9>([&](auto Pi) {
    constexpr int a = 2 * decltype(Pi)::value + 1, b = a + 1;
    const C cu = cdot<a, C>(m.ux, m.uy, m.uz);
    const C q = C(4.5) * cu * cu - m.usq;
    const C even = (a <= 6) ? wd1 + wr1 * q : wd2 + wr2 * q;
    const C odd = ((a <= 6) ? w3r1 : w3r2) * cu;
    const C sa = g[a] + omega * ((even + odd) - g[a]);
    const C sb = g[b] + omega * ((even - odd) - g[b]);
    if constexpr (ODD) {
      // The store to (x + c_a, a) hits the address the load of direction
      // opp(a) used; re-reading the offset from shared memory keeps the
      // compiler from holding all 18 64-bit addresses live across the update.
      S* pa = P + a * np + x + lds_volatile(dsc + a - 1);
      S* pb = P + b * np + x + lds_volatile(dsc + b - 1);
      Cd::st(pa, a, sa);
      Cd::st(pb, b, sb);
      chk_count(chk, P, pa, kQ * np, err);
      chk_count(chk, P, pb, kQ * np, err);
    } else {
      Cd::st(P + b * np + x, a, sa);
      Cd::st(P + a * np + x, b, sb);
      chk_count(chk, P, P + b * np + x, kQ * np, err);
      chk_count(chk, P, P + a * np + x, kQ * np, err);
    }
  });
  return m.drho;
}

// --------------------------------------------------- two sites per lane
// The bulk update of two z-adjacent sites x, x + 1 (x even) by one lane, for
// the FP32 and 16-bit storages: both sites share the tile's neighbour offsets,
// so one address serves both; a direction whose offset is even reads (and
// writes) the two values as one aligned 32-bit (16-bit storage) or 64-bit
// (FP32) word, an odd offset as two scalars; the collision runs on packed
// pairs with the two-wide FP32 instructions (add/sub/mul/fma .f32x2), so each
// floating-point instruction serves both sites.  The arithmetic is that of
// bulk_update, with the reciprocal of rho from the hardware approximation.
struct F2 {
  unsigned long long v;  // low word: site x, high word: site x + 1
};
__device__ __forceinline__ F2 mk2(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ F2 bc2(float a) { return mk2(a, a); }
__device__ __forceinline__ void split2(F2 a, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a.v));
}
__device__ __forceinline__ F2 add2(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 sub2(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 mul2(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {  // a b + c
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}
__device__ __forceinline__ float rcp_approx(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// Pair codecs: ld_al / st_al move the aligned word holding sites (x, x + 1);
// ld_un / st_un move the two elements one by one.  Conversions round as the
// single-site codecs do (to nearest even).
template <class S>
struct Codec2;
template <>
struct Codec2<float> {
  static __device__ __forceinline__ F2 ld_al(const float* p) {
    F2 r;
    r.v = *reinterpret_cast<const unsigned long long*>(p);
    return r;
  }
  static __device__ __forceinline__ F2 ld_un(const float* p) { return mk2(p[0], p[1]); }
  static __device__ __forceinline__ void st_al(float* p, F2 g) {
    *reinterpret_cast<unsigned long long*>(p) = g.v;
  }
  static __device__ __forceinline__ void st_un(float* p, F2 g) {
    float l, h;
    split2(g, l, h);
    p[0] = l;
    p[1] = h;
  }
};
// 16-bit pairs also travel as packed words (low half: the first site): two
// sites' values in one register from the load until the collision needs them.
__device__ __forceinline__ uint32_t ld_word(const void* p) { return ld_pop_b32(p); }
__device__ __forceinline__ uint32_t ld_u16(const void* p) { return ld_pop_u16(p); }
__device__ __forceinline__ uint32_t pack_u16(uint32_t lo, uint32_t hi) {
  return __byte_perm(lo, hi, 0x5410);
}
// An opaque copy: the compiler cannot tie the value read back after the
// moments to the one unpacked for them, so it keeps the packed word, not
// the two unpacked floats, live through the collision.
__device__ __forceinline__ uint32_t opaque(uint32_t v) {
  uint32_t r;
  asm volatile("mov.b32 %0, %1;" : "=r"(r) : "r"(v));
  return r;
}

template <>
struct Codec2<__half> {
  static __device__ __forceinline__ F2 unpack(uint32_t w) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return mk2(f.x, f.y);
  }
  static __device__ __forceinline__ F2 ld_al(const __half* p) { return unpack(ld_pop_b32(p)); }
  static __device__ __forceinline__ F2 ld_un(const __half* p) {
    return unpack(pack_u16(ld_pop_u16(p), ld_pop_u16(p + 1)));
  }
  static __device__ __forceinline__ void st_al(__half* p, F2 g) {
    float l, h;
    split2(g, l, h);
    uint32_t w;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(h), "f"(l));
    *reinterpret_cast<uint32_t*>(p) = w;
  }
  static __device__ __forceinline__ void st_un(__half* p, F2 g) {
    float l, h;
    split2(g, l, h);
    p[0] = __float2half_rn(l);
    p[1] = __float2half_rn(h);
  }
};
template <>
struct Codec2<__nv_bfloat16> {
  static __device__ __forceinline__ F2 unpack(uint32_t w) {
    return mk2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
  }
  static __device__ __forceinline__ F2 ld_al(const __nv_bfloat16* p) { return unpack(ld_pop_b32(p)); }
  static __device__ __forceinline__ F2 ld_un(const __nv_bfloat16* p) {
    const uint32_t a = ld_pop_u16(p), b = ld_pop_u16(p + 1);
    return mk2(__uint_as_float(a << 16), __uint_as_float(b << 16));
  }
  static __device__ __forceinline__ void st_al(__nv_bfloat16* p, F2 g) {
    float l, h;
    split2(g, l, h);
    uint32_t w;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(h), "f"(l));
    *reinterpret_cast<uint32_t*>(p) = w;
  }
  static __device__ __forceinline__ void st_un(__nv_bfloat16* p, F2 g) {
    float l, h;
    split2(g, l, h);
    p[0] = __float2bfloat16_rn(l);
    p[1] = __float2bfloat16_rn(h);
  }
};

template <class S>
__device__ __forceinline__ void chk_count2(int* chk, const S* P0, const S* p, int64_t lim,
                                           int* err) {
  chk_count(chk, P0, p, lim, err);
  chk_count(chk, P0, p + 1, lim, err);
}

// The collision of bulk_update for two sites at once, on packed pairs: gm(j)
// gives the pre-collision values for the moments, gp(j) the same values again
// for the relaxation (the 16-bit paths unpack them twice from packed words
// rather than hold 38 floats); store0(g*_0) receives the rest population and
// store<a, b>(g*_a, g*_b) those of each opposite pair (a odd, b = a + 1).
template <class GetM, class GetP, class St0, class St>
__device__ __forceinline__ F2 collide2(GetM&& gm, GetP&& gp, F2 omega, int* err_lo,
                                       int* err_hi, St0&& store0, St&& store) {
  // Eqs. (Density), (Momentum), grouped as in moments()
  F2 g[kQ];
  unroll<kQ>([&](auto J) {
    constexpr int j = decltype(J)::value;
    g[j] = gm(j);
  });
  const F2 a1 = sub2(g[1], g[2]), a3 = sub2(g[3], g[4]), a5 = sub2(g[5], g[6]);
  const F2 a7 = sub2(g[7], g[8]), a9 = sub2(g[9], g[10]), a11 = sub2(g[11], g[12]);
  const F2 a13 = sub2(g[13], g[14]), a15 = sub2(g[15], g[16]), a17 = sub2(g[17], g[18]);
  const F2 drho =
      add2(add2(add2(add2(g[0], add2(g[1], g[2])), add2(add2(g[3], g[4]), add2(g[5], g[6]))),
                add2(add2(add2(g[7], g[8]), add2(g[9], g[10])),
                     add2(add2(g[11], g[12]), add2(g[13], g[14])))),
           add2(add2(g[15], g[16]), add2(g[17], g[18])));
  const F2 jx = add2(add2(add2(a1, a7), add2(a9, a11)), a13);
  const F2 jy = add2(sub2(add2(a3, a7), sub2(a9, a15)), a17);
  const F2 jz = sub2(sub2(add2(a5, a11), sub2(a13, a15)), a17);
  const F2 rho = add2(bc2(1.0f), drho);
  float r0, r1;
  split2(rho, r0, r1);
  if (unstable(r0)) atomicOr(err_lo, kErrUnstable);
  if (unstable(r1)) atomicOr(err_hi, kErrUnstable);
  float d0, d1;
  split2(drho, d0, d1);
  const F2 inv = mk2(inv_one_plus(d0, r0, rcp_approx(r0)), inv_one_plus(d1, r1, rcp_approx(r1)));
  const F2 ux = mul2(jx, inv), uy = mul2(jy, inv), uz = mul2(jz, inv);
  const F2 usq = mul2(bc2(1.5f), fma2(uz, uz, fma2(uy, uy, mul2(ux, ux))));
  // rest population: g*_0 = g_0 + omega (w_0 (drho - rho usq) - g_0)
  const F2 e0 = mul2(bc2(1.0f / 3.0f), sub2(drho, mul2(rho, usq)));
  {
    const F2 g0 = gp(0);
    store0(fma2(omega, sub2(e0, g0), g0));
  }
  // opposite pairs (a, b): g^eq = even +- odd (see bulk_update)
  const F2 wd1 = mul2(drho, bc2(1.0f / 18.0f)), wd2 = mul2(drho, bc2(1.0f / 36.0f));
  const F2 wr1 = mul2(rho, bc2(1.0f / 18.0f)), wr2 = mul2(rho, bc2(1.0f / 36.0f));
  const F2 w3r1 = mul2(rho, bc2(3.0f / 18.0f)), w3r2 = mul2(rho, bc2(3.0f / 36.0f));
  const F2 nusq = sub2(bc2(0.0f), usq);
  unroll<9>([&](auto Pi) {
    constexpr int a = 2 * decltype(Pi)::value + 1;
    constexpr int pp = (a + 1) / 2;
    F2 cu;
    if constexpr (pp == 1) cu = ux;
    else if constexpr (pp == 2) cu = uy;
    else if constexpr (pp == 3) cu = uz;
    else if constexpr (pp == 4) cu = add2(ux, uy);
    else if constexpr (pp == 5) cu = sub2(ux, uy);
    else if constexpr (pp == 6) cu = add2(ux, uz);
    else if constexpr (pp == 7) cu = sub2(ux, uz);
    else if constexpr (pp == 8) cu = add2(uy, uz);
    else cu = sub2(uy, uz);
    const F2 q = fma2(mul2(bc2(4.5f), cu), cu, nusq);
    const F2 even = (a <= 6) ? fma2(wr1, q, wd1) : fma2(wr2, q, wd2);
    const F2 odd = mul2((a <= 6) ? w3r1 : w3r2, cu);
    const F2 ga = gp(a), gb = gp(a + 1);
    const F2 sa = fma2(omega, sub2(add2(even, odd), ga), ga);
    const F2 sb = fma2(omega, sub2(sub2(even, odd), gb), gb);
    store(std::integral_constant<int, a>{}, sa, sb);
  });
  return drho;
}

// The sum of a packed pair's two halves.
__device__ __forceinline__ float sum2(F2 a) {
  float lo, hi;
  split2(a, lo, hi);
  return lo + hi;
}

// Branch-free update of the sites x, x + 1 (x even) whose 18 links are fluid,
// both with the neighbour offsets dsc: one address per direction for both
// sites, packed loads and stores where the offset is even.
template <class S, bool ODD>
__device__ __forceinline__ float bulk_update2(S* P, int64_t np, int64_t x, const int32_t* dsc,
                                              float omega, int* err, int* chk) {
  using Cd = Codec2<S>;
  constexpr bool kPacked = sizeof(S) == 2;
  F2 g[kPacked ? 1 : kQ];
  uint32_t r[kPacked ? kQ : 1];
  unroll<kQ>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int o = dir_opp(j);
    const S* q;
    bool un = false;
    if constexpr (!ODD || j == 0) {
      q = P + j * np + x;
    } else {
      const int32_t dd = dsc[o - 1];
      q = P + o * np + x + dd;
      un = dd & 1;
    }
    if constexpr (kPacked) r[j] = un ? pack_u16(ld_u16(q), ld_u16(q + 1)) : ld_word(q);
    else g[j] = un ? Cd::ld_un(q) : Cd::ld_al(q);
  });
  auto gm = [&](int j) -> F2 {
    if constexpr (kPacked) return Cd::unpack(r[j]);
    else return g[j];
  };
  auto gp = [&](int j) -> F2 {
    if constexpr (kPacked) return Cd::unpack(opaque(r[j]));
    else return g[j];
  };
  return sum2(collide2(
      gm, gp, bc2(omega), err, err,
      [&](F2 s0) {
        Cd::st_al(P + x, s0);
        chk_count2(chk, P, P + x, kQ * np, err);
      },
      [&](auto A, F2 sa, F2 sb) {
        constexpr int a = decltype(A)::value, b = a + 1;
        if constexpr (ODD) {
          const int32_t da = lds_volatile(dsc + a - 1), db = lds_volatile(dsc + b - 1);
          S* pa = P + a * np + x + da;
          S* pb = P + b * np + x + db;
          if (da & 1) Cd::st_un(pa, sa);
          else Cd::st_al(pa, sa);
          if (db & 1) Cd::st_un(pb, sb);
          else Cd::st_al(pb, sb);
          chk_count2(chk, P, pa, kQ * np, err);
          chk_count2(chk, P, pb, kQ * np, err);
        } else {
          Cd::st_al(P + b * np + x, sa);
          Cd::st_al(P + a * np + x, sb);
          chk_count2(chk, P, P + b * np + x, kQ * np, err);
          chk_count2(chk, P, P + a * np + x, kQ * np, err);
        }
      }));
}

// Branch-free update of site xa of one bulk tile and site xb of another tile of
// the same lattice (the same lane of both), with their offsets da and db.
// SAME: the second tile directly follows the first with the same offsets, so
// each of its addresses is the first tile's plus one tile (an immediate
// offset, no second address).
template <class S, bool ODD, bool SAME>
__device__ __forceinline__ float bulk_update2v(S* P, int64_t np, int64_t xa, int64_t xb,
                                              const int32_t* da, const int32_t* db, float omega,
                                              int* err, int* chk) {
  using Cd = Codec<S>;
  constexpr bool kPacked = sizeof(S) == 2;
  F2 g[kPacked ? 1 : kQ];
  uint32_t r[kPacked ? kQ : 1];
  unroll<kQ>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int o = dir_opp(j);
    const S *qa, *qb;
    if constexpr (!ODD || j == 0) {
      qa = P + j * np + xa;
      qb = SAME ? qa + kTile : P + j * np + xb;
    } else {
      qa = P + o * np + xa + da[o - 1];
      qb = SAME ? qa + kTile : P + o * np + xb + db[o - 1];
    }
    if constexpr (kPacked) r[j] = pack_u16(ld_u16(qa), ld_u16(qb));
    else g[j] = mk2(Cd::ld(qa, j), Cd::ld(qb, j));
  });
  auto gm = [&](int j) -> F2 {
    if constexpr (kPacked) return Codec2<S>::unpack(r[j]);
    else return g[j];
  };
  auto gp = [&](int j) -> F2 {
    if constexpr (kPacked) return Codec2<S>::unpack(opaque(r[j]));
    else return g[j];
  };
  auto put = [&](S* pa, S* pb, F2 v, int i) {
    float lo, hi;
    split2(v, lo, hi);
    Cd::st(pa, i, lo);
    Cd::st(pb, i, hi);
    chk_count(chk, P, pa, kQ * np, err);
    chk_count(chk, P, pb, kQ * np, err);
  };
  return sum2(collide2(
      gm, gp, bc2(omega), err, err,
      [&](F2 s0) { put(P + xa, SAME ? P + xa + kTile : P + xb, s0, 0); },
      [&](auto A, F2 sa, F2 sb) {
        constexpr int i = decltype(A)::value, k = i + 1;  // the pair (i, k = opp i)
        if constexpr (ODD) {
          S* pi = P + i * np + xa + lds_volatile(da + i - 1);
          S* pk = P + k * np + xa + lds_volatile(da + k - 1);
          S* qi = SAME ? pi + kTile : P + i * np + xb + lds_volatile(db + i - 1);
          S* qk = SAME ? pk + kTile : P + k * np + xb + lds_volatile(db + k - 1);
          put(pi, qi, sa, i);
          put(pk, qk, sb, k);
        } else {
          S* pk = P + k * np + xa;
          S* pi = P + i * np + xa;
          put(pk, SAME ? pk + kTile : P + k * np + xb, sa, i);
          put(pi, SAME ? pi + kTile : P + i * np + xb, sb, k);
        }
      }));
}

// Update of a site of a boundary tile.  `code[i]` holds the tile's uniform
// offsets / non-fluid codes; irregular tiles use the staged per-site table.
// Pre-collision populations of a boundary site: direction j comes from its own
// slot when the link opp(j) leaves the fluid (bit opp(j) of `nf`), else (odd
// steps) from the neighbour along opp(j).
template <class S, bool ODD>
__device__ __forceinline__ void boundary_load(const S* P, int64_t np, int64_t x, uint32_t nf,
                                              const int32_t* dsc, bool irr, const int32_t* nbr_s,
                                              int lane, typename Codec<S>::C (&g)[kQ],
                                              int64_t n, int* err) {
  using Cd = Codec<S>;
  unroll<kQ>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int o = dir_opp(j);
    if constexpr (!ODD || j == 0) {
      g[j] = Cd::ld(P + j * np + x, j);
    } else {
      if ((nf >> o) & 1u) {
        g[j] = Cd::ld(P + j * np + x, j);
      } else {
        int64_t y = irr ? (int64_t)nbr_s[(o - 1) * kTile + lane] : x + dsc[o - 1];
        if (!chk_site(y, n, err)) y = x;  // checked builds: flagged, read a safe slot
        g[j] = Cd::ld(P + o * np + y, j);
      }
    }
  });
}

// Per-warp shared-memory area of the boundary kernels, in compute-type units:
// rows 0..18 the parked populations g, rows 19..24 the lanes' iolet states,
// then [5][32] doubles of per-site data (F, kappa/3, inlet profile p0, ps, pc).
template <class C>
struct BoundaryArea {
  static constexpr int size = 25 * kTile + 5 * kTile * (int)(sizeof(double) / sizeof(C));
};
constexpr int kAreaIolet = 19;  // first row of the iolet states

// Fused diagnostics: the momentum rho u of a site with iolet links, at its
// place among the lanes of the tiles that have such sites, for the fluxes.
template <class C>
__device__ __forceinline__ void diag_momentum(const DevLattice& d, int64_t slot, const Mom<C>& m) {
  const int64_t q = (int64_t)__ldg(d.diag_iotile + (slot >> 5)) * kTile + (slot & (kTile - 1));
  const int64_t js = d.diag_jstride;
  d.diag_j[q] = (double)(m.rho * m.ux);
  d.diag_j[js + q] = (double)(m.rho * m.uy);
  d.diag_j[2 * js + q] = (double)(m.rho * m.uz);
}
constexpr int kAreaSite = 25;   // first row (compute-type units) of the per-site doubles

// Update of a boundary site whose iolet links (if any) all lead to one iolet,
// without branches that differ between lanes: every direction does one load
// and one store, and each store's value and address are selected.
//   Loads: direction j from the site's own slot when the link opp(j) leaves
//     the fluid, else (odd steps) from the neighbour along opp(j).
//   Collision in the pair form of bulk_update: for each opposite pair (a, b)
//     the even and odd parts of the equilibrium give g^eq_a, g^eq_b and the
//     post-collision g*_a, g*_b.
//   Link i of the pair leaving the fluid (j = opp i, the other direction of the
//     same pair): half-way bounce-back stores g*_i into (x, j); the GZS form
//     stores f^eq_j(rho_b, u_b) + (1 - 1/tau) (g_j - g^eq_j) into (x, j), with
//     (rho_b, u_b) = (rho, U_w) at a wall link - whose equilibrium parts are
//     those of (rho, u) with c.u scaled by U_w/u_f = sw - and the site's iolet
//     state at an iolet link: (rho, u_in) at a velocity inlet, (rho_out, u) at a
//     density outlet.  A fluid link i streams g*_i: into (x, j) on even steps,
//     into (x + c_i, i) on odd steps.
// warp_io / warp_wall (warp-uniform): some lane of the tile has iolet links /
// elastic wall links, so their equilibria are computed at all; warp_nf: the
// union of the tile's non-fluid directions (pairs no lane needs skip the
// boundary values); site: the
// warp's [5][32] per-site F, kappa/3, p0, ps, pc (copies in flight until
// cp_async_wait_all); area: the warp's shared-memory area (BoundaryArea).
// The odd-step slot deltas (opp(i) - i) np below stay within one row length
// because opposite directions are numbered next to each other.
constexpr bool opposites_adjacent() {
  for (int i = 1; i < kQ; ++i)
    if (dir_opp(i) - i != 1 && dir_opp(i) - i != -1) return false;
  return true;
}
static_assert(opposites_adjacent(), "opposite directions must be adjacent");

template <class S, bool ODD>
__device__ __forceinline__ typename Codec<S>::C boundary_fast(const DevLattice& d,
                                                              const StepParams& p,
                                              typename Codec<S>::C omega, S* P, int64_t x,
                                              const int32_t* offp, int ostride, uint32_t smask,
                                              uint32_t iom, const double* site,
                                              const int32_t* nbr_s, int lane, int64_t slot,
                                              bool warp_io, bool warp_wall, uint32_t warp_nf,
                                              typename Codec<S>::C* area) {
  using Cd = Codec<S>;
  using C = typename Cd::C;
  const int64_t np = d.npad;
  const uint32_t nf = smask & kDirBits;
  // Odd steps: the offset nbr(x, i) - x of a fluid link i is offp[(i - 1)
  // ostride] (the tile's or the lane's segment's offsets with stride 1, or the
  // lane's column of the staged per-site rows with stride 32), read the same
  // way in every case, and the choice between the site's own slot and the
  // neighbour's is a select, not a branch.
  auto off = [&](int i) -> int32_t { return offp[(i - 1) * ostride]; };
  // the same offset re-read at store time (volatile: not held in registers
  // from the loads to the stores)
  auto off_again = [&](int i) -> int32_t { return lds_volatile(offp + (i - 1) * ostride); };
  // Odd steps: link i's slot is A_i = P + i np + x + delta_i, with delta_i =
  // nbr(x, i) - x when the link is fluid and (opp(i) - i) np = +-np when it
  // leaves the fluid (the site's own slot of direction opp(i)).  The load of
  // g_opp(i) and the store of the post-collision value of direction i both
  // use A_i.  In 32-bit parts (x < 2^32, |delta_i| < 2^31 since npad < 2^31)
  // each address is two wide multiply-adds on the row base i np, which does
  // not depend on the lane.
  const int32_t np32 = (int32_t)np;
  auto delta = [&](int i, int32_t off_i) -> int32_t {
    const bool fluid = !((nf >> i) & 1u);
    int32_t dl = fluid ? off_i : (dir_opp(i) - i) * np32;
    // checked builds: a bad neighbour index is flagged and the own slot used
    if (kChecked && fluid && !chk_site(x + off_i, d.n, d.err)) dl = (dir_opp(i) - i) * np32;
    return dl;
  };
  auto slot_at = [&](int i, uint32_t xs, int32_t dl) -> S* {
    return P + (int64_t)i * np + xs + dl;
  };
  C g[kQ];
  unroll<kQ>([&](auto J) {
    constexpr int j = decltype(J)::value;
    constexpr int o = dir_opp(j);
    if constexpr (!ODD || j == 0) {
      g[j] = Cd::ld(P + j * np + x, j);
    } else {
      g[j] = Cd::ld(slot_at(o, (uint32_t)x, delta(o, off(o))), j);
    }
  });
  const Mom<C> m = moments(g);
  // FP32 compute: g stays in registers through the boundary rule (at 72
  // registers no spills; parking it in shared memory and reading it back
  // pair by pair, needed at 64, measured 1.5-3 % slower).  FP64: g is parked
  // in the warp's area and read back pair by pair (volatile, so the 19
  // doubles are not held in registers through the rule).
  constexpr bool kPark = std::is_same<C, double>::value;
  if constexpr (kPark) {
    unroll<kQ>([&](auto J) {
      constexpr int j = decltype(J)::value;
      area[j * kTile + lane] = g[j];
    });
  }
  auto gv = [&](int j) -> C {
    if constexpr (kPark) return static_cast<const volatile C*>(area)[j * kTile + lane];
    else return g[j];
  };
  if (unstable(m.rho)) atomicOr(d.err, kErrUnstable);
  const C keep = C(1) - omega;  // (1 - 1/tau)
  // Elastic wall (Sec. 2.3-2.4): dE in FP64, the ratio sw = U_w/u_f =
  // (F + dr - dx)/dr with dr = dx + dE in the compute type.
  C sw = C(0);
  if ((smask & kHasWall) && p.elastic) {
    cp_async_wait_all();
    // F (compute type), kappa c_s^2 (FP64)
    const C Fw = reinterpret_cast<const C*>(site)[lane];
    const double Kw = site[kTile + lane];
    const double dE = tube_law(Kw, m.rho, p);
    if constexpr (std::is_same<C, double>::value) {
      const double dr = 1.0 + dE;
      sw = (Fw + dr - 1.0) / dr;
    } else {
      const float e = (float)dE;
      sw = (Fw + e) * recip(1.0f + e);
    }
    if (p.write_state) {
      const int64_t ss = d.slot_stride;
      d.slot_dE[slot] = dE;
      d.slot_Uw[slot] = (double)(sw * m.ux);
      d.slot_Uw[ss + slot] = (double)(sw * m.uy);
      d.slot_Uw[2 * ss + slot] = (double)(sw * m.uz);
    }
  }
  const C sw2 = sw * sw;
  // The site's iolet state (rho_b, u_b): velocity inlet (Sec. 3) u_in =
  // a (u_mean p0 + u_amp (ps sin th + pc cos th)) with rho_b = rho; density
  // outlet rho_b = rho_out with u_b = u.  Parked in the warp's shared-memory
  // area (read back only by tiles with iolet links), not held in registers.
  if (warp_io) {
  C rb = m.rho, drb = m.drho, ubx = m.ux, uby = m.uy, ubz = m.uz, usqb = m.usq;
  if (iom & kDirBits) {
    const int k = (int)((iom & kIoletIdBits) >> kIoletShift);
    const IoletDev& io = d.iolets[k];
    if (io.kind == LBM_IOLET_VELOCITY) {
      cp_async_wait_all();
      // rows 2..4 of the per-site area: p0, ps, pc in the compute type
      const C pr0 = reinterpret_cast<const C*>(site + 2 * kTile)[lane];
      const C pr1 = reinterpret_cast<const C*>(site + 3 * kTile)[lane];
      const C pr2 = reinterpret_cast<const C*>(site + 4 * kTile)[lane];
      const int64_t step = p.step + (p.step_dev ? *p.step_dev : 0);
      inlet_velocity(io, step, pr0, pr1, pr2, ubx, uby, ubz);
      usqb = C(1.5) * (ubx * ubx + uby * uby + ubz * ubz);
    } else {
      outlet_density(io, rb, drb);
    }
  }
  C* iost = area + kAreaIolet * kTile;
  iost[0 * kTile + lane] = rb;
  iost[1 * kTile + lane] = drb;
  iost[2 * kTile + lane] = ubx;
  iost[3 * kTile + lane] = uby;
  iost[4 * kTile + lane] = ubz;
  iost[5 * kTile + lane] = usqb;
  }
  // rest population: stays at x
  {
    const C g0 = gv(0);
    Cd::st(P + x, 0, g0 + omega * (geq<0, C>(m.drho, m.rho, m.ux, m.uy, m.uz, m.usq) - g0));
  }
  chk_count(d.chk, P, P + x, kQ * np, d.err);
  const bool bounce = !p.elastic;
  // Store addresses from a base and a stride (even steps) or a site index
  // (odd steps) the compiler cannot identify with those of the loads (opaque
  // copies): otherwise it keeps the 19 load addresses, or the rows' offsets,
  // live until the stores that reuse them.
  S* Pst;
  asm volatile("mov.b64 %0, %1;" : "=l"(Pst) : "l"(P));
  uint32_t xst;
  asm volatile("mov.b32 %0, %1;" : "=r"(xst) : "r"((uint32_t)x));
  unroll<9>([&](auto Pi) {
    constexpr int a = 2 * decltype(Pi)::value + 1, b = a + 1;
    constexpr C w = a <= 6 ? C(1.0 / 18.0) : C(1.0 / 36.0);
    const C cu = cdot<a, C>(m.ux, m.uy, m.uz);
    const C wr = m.rho * w;
    const C wrq = wr * (C(4.5) * cu * cu - m.usq);
    const C wd = m.drho * w;
    const C even = wd + wrq;
    const C odd = C(3) * wr * cu;
    const C eqa = even + odd, eqb = even - odd;
    const C ga = gv(a), gb = gv(b);
    const C sa = ga + omega * (eqa - ga);
    const C sb = gb + omega * (eqb - gb);
    // the pair's links leave the fluid at some lane of the tile (warp-uniform)
    const bool pair_nf = (warp_nf >> a) & 3u;
    // GZS values of the pair's two directions at a wall: f^eq(rho, sw u) parts
    C wa = C(0), wb = C(0);
    if (warp_wall && pair_nf) {
      const C evw = wd + sw2 * wrq, odw = sw * odd;
      wa = evw + odw + keep * (ga - eqa);
      wb = evw - odw + keep * (gb - eqb);
    }
    // ... and at the site's iolet
    C ia = C(0), ib = C(0);
    if (warp_io && pair_nf) {
      const C* iost = area + kAreaIolet * kTile;
      const C rb = iost[0 * kTile + lane], drb = iost[1 * kTile + lane];
      const C cub = cdot<a, C>(iost[2 * kTile + lane], iost[3 * kTile + lane],
                               iost[4 * kTile + lane]);
      const C evb = w * (drb + rb * (C(4.5) * cub * cub - iost[5 * kTile + lane]));
      const C odb = w * C(3) * rb * cub;
      ia = evb + odb + keep * (ga - eqa);
      ib = evb - odb + keep * (gb - eqb);
    }
    // link a (store into direction b's slot when it leaves the fluid) and link b
    const bool nfa = (nf >> a) & 1u, nfb = (nf >> b) & 1u;
    const bool ioa = (iom >> a) & 1u, iob = (iom >> b) & 1u;
    const C va = nfa ? (ioa ? ib : (bounce ? sa : wb)) : sa;
    const C vb = nfb ? (iob ? ia : (bounce ? sb : wa)) : sb;
    S* pa;
    S* pb;
    if constexpr (ODD) {
      pa = slot_at(a, xst, delta(a, off_again(a)));
      pb = slot_at(b, xst, delta(b, off_again(b)));
    } else {
      pa = Pst + b * np + x;
      pb = Pst + a * np + x;
    }
    Cd::st(pa, nfa ? b : a, va);
    Cd::st(pb, nfb ? a : b, vb);
    chk_count(d.chk, P, pa, kQ * np, d.err);
    chk_count(d.chk, P, pb, kQ * np, d.err);
  });
  if (p.diag && (iom & kDirBits)) diag_momentum(d, slot, m);
  return m.drho;
}

// D3Q19 vectors and weights for directions known only at run time (the
// boundary rule loops over the links that leave the fluid), computed from bit
// masks of the directions with c = +1 and c = -1 in each axis: no table, so
// lanes asking for different directions do not serialise on a memory port.
template <int (*F)(int)>
__host__ __device__ constexpr uint32_t dir_mask(int v) {
  uint32_t m = 0;
  for (int i = 0; i < kQ; ++i)
    if (F(i) == v) m |= 1u << i;
  return m;
}
template <class C>
__device__ __forceinline__ C dir_component(uint32_t plus, uint32_t minus, int i) {
  return C((int)((plus >> i) & 1u) - (int)((minus >> i) & 1u));
}
template <class C>
__device__ __forceinline__ void dir_vec(int i, C& cx, C& cy, C& cz) {
  cx = dir_component<C>(dir_mask<dir_x>(1), dir_mask<dir_x>(-1), i);
  cy = dir_component<C>(dir_mask<dir_y>(1), dir_mask<dir_y>(-1), i);
  cz = dir_component<C>(dir_mask<dir_z>(1), dir_mask<dir_z>(-1), i);
}
template <class C>
__device__ __forceinline__ C dir_weight(int i) {
  return i == 0 ? C(1.0 / 3.0) : (i <= 6 ? C(1.0 / 18.0) : C(1.0 / 36.0));
}

// Collision, boundary rule and stores of a boundary site with pre-collision
// populations g.  smask, iom: the site's link masks; Fw, Kw: its wall
// parameters; pr0..pr2: its inlet profile (p0, ps, pc); nbr_s: the staged
// per-site neighbour rows (irregular tiles on odd steps); gsm: the warp's
// [19][32] shared-memory area where g is parked for the boundary rule.
template <class S, bool ODD>
__device__ __forceinline__ typename Codec<S>::C boundary_update(const DevLattice& d,
                                                                const StepParams& p,
                                                typename Codec<S>::C omega, S* P,
                                                int64_t x, const int32_t* dsc, bool irr,
                                                uint32_t smask, uint32_t iom,
                                                typename Codec<S>::C Fw, double Kw,
                                                typename Codec<S>::C pr0, typename Codec<S>::C pr1,
                                                typename Codec<S>::C pr2,
                                                const int32_t* nbr_s, int lane, int64_t slot,
                                                typename Codec<S>::C (&g)[kQ],
                                                typename Codec<S>::C* gsm) {
  using Cd = Codec<S>;
  using C = typename Cd::C;
  const int64_t np = d.npad;
  const Mom<C> m = moments(g);
  if (unstable(m.rho)) atomicOr(d.err, kErrUnstable);
  const C keep = C(1) - omega;  // (1 - 1/tau)
  // neighbour index of a fluid link i (odd steps)
  auto nb = [&](int i) -> int64_t {
    return irr ? (int64_t)nbr_s[(i - 1) * kTile + lane] : x + dsc[i - 1];
  };
  // Rest population and the links that stay in the fluid: stream f*.
  Cd::st(P + x, 0, g[0] + omega * (geq<0, C>(m.drho, m.rho, m.ux, m.uy, m.uz, m.usq) - g[0]));
  chk_count(d.chk, P, P + x, kQ * np, d.err);
  unroll<kQ - 1>([&](auto I0) {
    constexpr int i = decltype(I0)::value + 1;
    if (!((smask >> i) & 1u)) {
      const C si = g[i] + omega * (geq<i, C>(m.drho, m.rho, m.ux, m.uy, m.uz, m.usq) - g[i]);
      S* pi;
      if constexpr (ODD) {
        const int64_t y = nb(i);
        if (!chk_site(y, d.n, d.err)) return;
        pi = P + i * np + y;
      } else {
        pi = P + dir_opp(i) * np + x;
      }
      Cd::st(pi, i, si);
      chk_count(d.chk, P, pi, kQ * np, d.err);
    }
  });
  if (p.diag && ((iom & kDirBits) || (smask & kMultiIolet))) diag_momentum(d, slot, m);
  uint32_t nf = smask & kDirBits;
  if (!nf) return m.drho;
  // Elastic wall (Sec. 2.3-2.4): the tube-law expansion dE in FP64, and the
  // ratio sw = U_w/u_f = (F + dr - dx)/dr with dr = dx + dE in the compute
  // type (FP64 throughput is low on this GPU and the ratio only scales an FP32
  // velocity on the FP32 paths).  U_w = sw u.
  C sw = C(0);
  if ((smask & kHasWall) && p.elastic) {
    // Kw holds kappa c_s^2 = kappa / 3, so dE = Kw max(0, rho - rho0)
    const double dE = tube_law(Kw, m.rho, p);
    if constexpr (std::is_same<C, double>::value) {
      const double dr = 1.0 + dE;
      sw = (Fw + dr - 1.0) / dr;
    } else {
      const float e = (float)dE;
      sw = mul_pin(Fw + e, recip(1.0f + e));
    }
    if (p.write_state) {
      const int64_t ss = d.slot_stride;
      d.slot_dE[slot] = dE;  // dE of this step; dr = 1 + dE
      d.slot_Uw[slot] = (double)(sw * m.ux);
      d.slot_Uw[ss + slot] = (double)(sw * m.uy);
      d.slot_Uw[2 * ss + slot] = (double)(sw * m.uz);
    }
  }
  // Inlet velocity (Sec. 3): u_in = a (u_mean p0 + u_amp (ps sin th + pc cos th)).
  C uix = C(0), uiy = C(0), uiz = C(0);
  if (smask & kHasInlet) {
    const int k = (int)((iom & kIoletIdBits) >> kIoletShift);
    const int64_t step = p.step + (p.step_dev ? *p.step_dev : 0);
    inlet_velocity(d.iolets[k], step, pr0, pr1, pr2, uix, uiy, uiz);
  }
  const C uisq = mul_pin(C(1.5), fma_pin(uiz, uiz, fma_pin(uiy, uiy, mul_pin(uix, uix))));
  // Links that leave the fluid: the population of direction j = opp(i) that
  // the site receives at the next step is rebuilt here and written to its own
  // slot (x, j) - half-way bounce-back f*_i, or the GZS form
  // f^eq_j(rho_b, u_b) + (1 - 1/tau) f^neq_j with (rho_b, u_b) = (rho, U_w) at a
  // wall, (rho, u_in) at a velocity inlet, (rho_out, u) at a density outlet.
  const int32_t io_code = -2 - (int32_t)((iom & kIoletIdBits) >> kIoletShift);
  // Boundary code of the non-fluid link i: -1 wall, -2-k iolet k.
  auto link_code = [&](int i) -> int32_t {
    if (smask & kMultiIolet)
      return (ODD && irr) ? nbr_s[(i - 1) * kTile + lane]
                          : __ldg(d.slot_nbr + (i - 1) * d.slot_stride + slot);
    return ((iom >> i) & 1u) ? io_code : -1;
  };
  // Value stored into (x, j) for the non-fluid link i = opp(j), from
  // cu = c_j . u, ci = c_j . u_in, the weight w_j and the pre-collision g_i, g_j.
  auto link_value = [&](int32_t c, C cu, C ci, C wj, C gi, C gj) -> C {
    const C quad = fma_pin(mul_pin(C(4.5), cu), cu, -m.usq);
    if (c == -1 && !p.elastic) {
      // f*_i, with c_i = -c_j
      const C ei = mul_pin(wj, fma_pin(m.rho, fma_pin(C(-3), cu, quad), m.drho));
      return fma_pin(omega, ei - gi, gi);
    }
    const C fneq = gj - mul_pin(wj, fma_pin(m.rho, fma_pin(C(3), cu, quad), m.drho));
    C e;
    if (c == -1) {
      // U_w = sw u: c_j . U_w = sw cu, 1.5 U_w^2 = sw^2 1.5 u^2
      const C inner = fma_pin(C(3), mul_pin(sw, cu), mul_pin(mul_pin(sw, sw), quad));
      e = mul_pin(wj, fma_pin(m.rho, inner, m.drho));
    } else {
      const IoletDev& io = d.iolets[-2 - c];
      if (io.kind == LBM_IOLET_VELOCITY) {
        const C inner = fma_pin(mul_pin(C(4.5), ci), ci, fma_pin(C(3), ci, -uisq));
        e = mul_pin(wj, fma_pin(m.rho, inner, m.drho));
      } else {
        C ro, dro;
        outlet_density(io, ro, dro);
        e = mul_pin(wj, fma_pin(ro, fma_pin(C(3), cu, quad), dro));
      }
    }
    return fma_pin(keep, fneq, e);
  };
  if (!(ODD && irr)) {
    // One branch per direction, so c_j, w_j and g are compile-time operands.
    // On coherent tiles (straight walls, iolet planes) every lane has the same
    // non-fluid links and the branches are uniform across the warp; on even
    // steps irregular tiles take this form too, which measured faster than
    // the loop below while no neighbour rows are staged.
    unroll<kQ - 1>([&](auto I0) {
      constexpr int i = decltype(I0)::value + 1;
      constexpr int j = dir_opp(i);
      if ((nf >> i) & 1u) {
        const C val = link_value(link_code(i), cdot<j, C>(m.ux, m.uy, m.uz),
                                 cdot<j, C>(uix, uiy, uiz), weight<C>(j), g[i], g[j]);
        Cd::st(P + j * np + x, j, val);
        chk_count(d.chk, P, P + j * np + x, kQ * np, d.err);
      }
    });
  } else {
    // Odd steps of irregular tiles: lanes differ in their non-fluid links,
    // so each lane loops over its own; g is parked in the warp's shared
    // memory and c_j, w_j come from the constant table.
    unroll<kQ>([&](auto J) {
      constexpr int j = decltype(J)::value;
      gsm[j * kTile + lane] = g[j];
    });
    while (nf) {
      const int i = __ffs(nf) - 1;
      nf &= nf - 1;
      const int j = dir_opp(i);
      C cx, cy, cz;
      dir_vec<C>(j, cx, cy, cz);
      const C cu = fma_pin(cz, m.uz, fma_pin(cy, m.uy, mul_pin(cx, m.ux)));
      const C ci = fma_pin(cz, uiz, fma_pin(cy, uiy, mul_pin(cx, uix)));
      const C val = link_value(link_code(i), cu, ci, dir_weight<C>(j), gsm[i * kTile + lane],
                               gsm[j * kTile + lane]);
      Cd::st(P + j * np + x, j, val);
      chk_count(d.chk, P, P + j * np + x, kQ * np, d.err);
    }
  }
  return m.drho;
}

// Sites linked to two or more iolets (each non-fluid link takes its own code
// from the neighbour table): loads and the per-link boundary rule, out of line
// so that its registers do not weigh on the common path.
template <class S, bool ODD>
__device__ __noinline__ void boundary_slow(const DevLattice& d, const StepParams& p, S* P,
                                           int64_t x, const int32_t* dsc, bool irr, uint32_t smask,
                                           uint32_t iom, typename Codec<S>::C Fw, double Kw,
                                           typename Codec<S>::C pr0, typename Codec<S>::C pr1,
                                           typename Codec<S>::C pr2, const int32_t* nbr_s, int lane,
                                           int64_t slot, typename Codec<S>::C* gsm) {
  using C = typename Codec<S>::C;
  C g[kQ];
  boundary_load<S, ODD>(P, d.npad, x, smask & kDirBits, dsc, irr, nbr_s, lane, g, d.n, d.err);
  boundary_update<S, ODD>(d, p, omega_as<C>(p.omega, p.omega_f), P, x, dsc, irr, smask, iom, Fw,
                          Kw, pr0, pr1, pr2, nbr_s, lane, slot, g, gsm);
}

#ifndef LBM_BULK_MINB
#define LBM_BULK_MINB 8
#endif
#ifndef LBM_BULK2_MINB
#define LBM_BULK2_MINB 6
#endif
#ifndef LBM_BULK2_MINB16
#define LBM_BULK2_MINB16 8
#endif
// Resident CTAs per SM requested of the bulk kernels with W warps per CTA: the
// same warps per SM whatever W (FP64: 16 warps; else LBM_BULK_MINB (one site
// per lane) or LBM_BULK2_MINB (two sites per lane) CTAs of 4 warps).
template <class S, int W>
struct BulkMinBlocks {
  static constexpr int one = sizeof(S) == 8 ? 16 / W : LBM_BULK_MINB * 4 / W;
  static constexpr int two_ctas = sizeof(S) == 2 ? LBM_BULK2_MINB16 : LBM_BULK2_MINB;
  static constexpr int two = two_ctas * 4 / W < 1 ? 1 : two_ctas * 4 / W;
};
// The ensemble kernels hold each member's pointers and strides in registers
// (a single lattice reads them from the kernel parameters), so they get their
// own register budgets, measured on the 256-tube ensemble: 80 registers for the
// one-site bulk kernel (FP32 +14 % over 64, which spill), 128 for the two-site
// bulk kernel (FP16S +11 % over 80), 72 for the boundary kernel (FP16S +7 %
// over 80, +2 % over 64).
#ifndef LBM_ENS_BULK_MINB
#define LBM_ENS_BULK_MINB 6
#endif
#ifndef LBM_ENS_BULK2_MINB
#define LBM_ENS_BULK2_MINB 4
#endif
#ifndef LBM_ENS_BOUNDARY_MINB
#define LBM_ENS_BOUNDARY_MINB 7
#endif
template <class S, int W>
struct EnsBulkMinBlocks {
  static constexpr int one = sizeof(S) == 8 ? 16 / W : LBM_ENS_BULK_MINB * 4 / W;
  static constexpr int two = LBM_ENS_BULK2_MINB * 4 / W < 1 ? 1 : LBM_ENS_BULK2_MINB * 4 / W;
};
#ifndef LBM_BOUNDARY_WARPS
#define LBM_BOUNDARY_WARPS 4
#endif
constexpr int kBoundaryWarps = LBM_BOUNDARY_WARPS;  // k_boundary: tiles (warps) per CTA

// Bulk tile at launch position k (whole warp); dsc: the warp's 20-word area.
// Returns the lane's rho - 1 (0 for a lane without a site).  With SLOT the
// tile's sum goes to *slot instead (fused diagnostics): from inside the update
// when every lane has a site (bulk tiles always do), else after it.
template <class S, bool ODD, bool SLOT = false>
__device__ __forceinline__ typename Codec<S>::C bulk_tile(const DevLattice& d,
                                                          const StepParams& p, int64_t k,
                                                          int32_t* dsc, int lane,
                                                          double* slot = nullptr) {
  using C = typename Codec<S>::C;
  // a warp that updates tiles in a loop (persistent kernel): every lane is done
  // with the previous tile's descriptor before it is overwritten
  __syncwarp();
  if (lane < 20) dsc[lane] = __ldg(reinterpret_cast<const int32_t*>(d.launch + k) + lane);
  if (p.prefetch > 0 && k + p.prefetch < d.n_tiles && lane < kQ) {
    const int64_t tp = __ldg(&d.launch[k + p.prefetch].tile);
    bulk_prefetch_l2(static_cast<const S*>(d.pop) + lane * d.npad + tp * kTile,
                     kTile * sizeof(S));
  }
  __syncwarp();
  const int64_t x = (int64_t)dsc[19] * kTile + lane;
  if constexpr (SLOT) {
    bool ok = x < d.n;
    if constexpr (kChecked && ODD)
      for (int o = 0; o < 18; ++o) ok = ok && chk_site(x + dsc[o], d.n, d.err);
    if (__all_sync(0xffffffffu, ok)) {
      bulk_update<S, ODD, true>(static_cast<S*>(d.pop), d.npad, x, dsc,
                                omega_as<C>(p.omega, p.omega_f), d.err, d.chk, slot);
      return C(0);
    }
    const C dr = ok ? bulk_update<S, ODD>(static_cast<S*>(d.pop), d.npad, x, dsc,
                                          omega_as<C>(p.omega, p.omega_f), d.err, d.chk)
                    : C(0);
    const C sum = warp_sum(dr);
    if (lane == 0) *slot = (double)sum;
    return C(0);
  }
  if (x >= d.n) return C(0);
  if constexpr (kChecked && ODD) {
    bool ok = true;
    for (int o = 0; o < 18; ++o) ok = chk_site(x + dsc[o], d.n, d.err) && ok;
    if (!ok) return C(0);
  }
  return bulk_update<S, ODD>(static_cast<S*>(d.pop), d.npad, x, dsc,
                             omega_as<C>(p.omega, p.omega_f), d.err, d.chk);
}


// The fields of a lattice the bulk kernels read (a member of an ensemble is
// read field by field from its device table, not copied whole).
struct BulkView {
  void* pop;
  const LaunchDesc* launch;
  int* err;
  int* chk;
  int64_t npad, n, n_tiles;
};
__device__ __forceinline__ BulkView bulk_view(const DevLattice& d) {
  return BulkView{d.pop, d.launch, d.err, d.chk, d.npad, d.n, d.n_tiles};
}

// Two bulk tiles per warp, two sites per lane (FP32 and 16-bit storage): tile
// A at launch position kA of lattice dA and, when `two`, tile B at launch
// position kB of lattice dB (the same lattice, or another member of an
// ensemble); omA, omB their relaxation rates; dsc2: the warp's two 20-word
// descriptor areas.
//   VERT = false: lanes 0..15 take tile A, lanes 16..31 tile B, lane l the
//     z-adjacent sites 2 (l mod 16), 2 (l mod 16) + 1 of its tile (packed words);
//   VERT = true: lane l takes site l of both tiles (scalar accesses; one
//     address for both when B directly follows A in the same lattice with the
//     same offsets).
// A site without a partner takes the single-site update.
template <class S, bool ODD, bool VERT>
__device__ __forceinline__ float bulk_pair_warp(const BulkView& dA, int64_t kA, float omA,
                                               const BulkView& dB, int64_t kB, float omB,
                                               bool two, bool one_lattice, int64_t prefetch,
                                               int32_t (*dsc2)[20], int lane) {
  if (lane < 20) {
    dsc2[0][lane] = __ldg(reinterpret_cast<const int32_t*>(dA.launch + kA) + lane);
    if (two) dsc2[1][lane] = __ldg(reinterpret_cast<const int32_t*>(dB.launch + kB) + lane);
  }
  if (prefetch > 0 && lane < kQ) {
    if (kA + prefetch < dA.n_tiles) {
      const int64_t tp = __ldg(&dA.launch[kA + prefetch].tile);
      bulk_prefetch_l2(static_cast<const S*>(dA.pop) + lane * dA.npad + tp * kTile,
                       kTile * sizeof(S));
    }
    if (two && kB + prefetch < dB.n_tiles) {
      const int64_t tp = __ldg(&dB.launch[kB + prefetch].tile);
      bulk_prefetch_l2(static_cast<const S*>(dB.pop) + lane * dB.npad + tp * kTile,
                       kTile * sizeof(S));
    }
  }
  __syncwarp();
  if constexpr (!VERT) {
    const int half = lane >> 4;
    if (half && !two) return 0.0f;
    // this half's lattice, field by field (no reference chosen at run time)
    S* P = static_cast<S*>(half ? dB.pop : dA.pop);
    const int64_t np = half ? dB.npad : dA.npad, n = half ? dB.n : dA.n;
    int* err = half ? dB.err : dA.err;
    int* chk = half ? dB.chk : dA.chk;
    const int32_t* dsc = dsc2[half];
    const int64_t x = (int64_t)dsc[19] * kTile + 2 * (lane & 15);
    if (x >= n) return 0.0f;
    if constexpr (kChecked && ODD) {
      bool ok = true;
      for (int o = 0; o < 18; ++o) ok = chk_site(x + dsc[o], n, err) && ok;
      if (x + 1 < n)
        for (int o = 0; o < 18; ++o) ok = chk_site(x + 1 + dsc[o], n, err) && ok;
      if (!ok) return 0.0f;
    }
    // a bulk tile is never the ragged last tile (its last site has a +x link
    // out of the fluid), so x + 1 < n; the guard keeps the update in bounds
    if (x + 1 < n) return bulk_update2<S, ODD>(P, np, x, dsc, half ? omB : omA, err, chk);
    return bulk_update<S, ODD>(P, np, x, dsc, half ? omB : omA, err, chk);
  } else {
    const int32_t* da = dsc2[0];
    const int64_t xa = (int64_t)da[19] * kTile + lane;
    S* PA = static_cast<S*>(dA.pop);
    if (!two) {
      if (xa < dA.n) return bulk_update<S, ODD>(PA, dA.npad, xa, da, omA, dA.err, dA.chk);
      return 0.0f;
    }
    const int32_t* db = dsc2[1];
    const int64_t xb = (int64_t)db[19] * kTile + lane;
    if (!one_lattice || xa >= dA.n || xb >= dA.n) {
      // the two tiles belong to different members of an ensemble (or a site
      // has no partner, not reached for bulk tiles): one site at a time
      S* PB = static_cast<S*>(dB.pop);
      float r = 0.0f;
      if (xa < dA.n) r += bulk_update<S, ODD>(PA, dA.npad, xa, da, omA, dA.err, dA.chk);
      if (xb < dB.n) r += bulk_update<S, ODD>(PB, dB.npad, xb, db, omB, dB.err, dB.chk);
      return r;
    }
    // B directly follows A with the same offsets (warp-uniform)
    const bool same = __all_sync(
        0xFFFFFFFFu, lane < 18 ? da[lane] == db[lane] : (lane == 18 ? db[19] == da[19] + 1 : true));
    if constexpr (kChecked && ODD) {
      bool ok = true;
      for (int o = 0; o < 18; ++o)
        ok = chk_site(xa + da[o], dA.n, dA.err) && chk_site(xb + db[o], dA.n, dA.err) && ok;
      if (!ok) return 0.0f;
    }
    if (same) return bulk_update2v<S, ODD, true>(PA, dA.npad, xa, xb, da, db, omA, dA.err, dA.chk);
    return bulk_update2v<S, ODD, false>(PA, dA.npad, xa, xb, da, db, omA, dA.err, dA.chk);
  }
}

// Bulk tiles of one lattice, two per warp (warp w of block b: the bulk tiles
// at launch positions n_boundary + 2 (b W + w) and the one after it).
// DIAG: also write the tiles' sums of rho - 1 (fused diagnostics), a separate
// instantiation so that ordinary steps keep their registers.
template <class S, bool ODD, bool VERT, int W, bool DIAG = false>
__global__ void __launch_bounds__(W * 32, BulkMinBlocks<S, W>::two)
    k_bulk2(const DevLattice d, const StepParams p) {
  __shared__ __align__(16) int32_t desc_s[W][2][20];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k0 = d.n_boundary + 2 * ((int64_t)blockIdx.x * W + w);
  if (k0 >= d.n_tiles) return;  // warp-uniform
  const BulkView v = bulk_view(d);
  const bool two = k0 + 1 < d.n_tiles;
  const float dr = bulk_pair_warp<S, ODD, VERT>(v, k0, p.omega_f, v, k0 + 1, p.omega_f, two, true,
                                                p.prefetch, desc_s[w], lane);
  if constexpr (DIAG) {
    // the two tiles' mass under the first one's launch position
    const float m = warp_sum(dr);
    if (lane == 0) d.diag_mass[k0] = (double)m;
    if (lane == 1 && two) d.diag_mass[k0 + 1] = 0.0;
  }
}

// Even steps of the 16-bit bulk tiles with staged rows (LBM_TUNE_BULK_SITES 5):
// a fixed grid of warps walks the bulk tile pairs.  While a warp updates one
// pair from shared memory, two TMA copies (one per tile, 19 rows x 32 sites
// of the row-major population array, described by the tensor map tm) bring
// the next pair into the other stage of its two-stage ring, each stage
// completing on its own mbarrier; even steps read each site's own slots, so
// every copy starts on a tile boundary.  No register holds a population in
// flight.  Lane l takes the adjacent sites 2 (l mod 16), 2 (l mod 16) + 1 of
// the first (l < 16) or second tile, as k_bulk2 does; a lone last tile takes
// bulk_tile.
constexpr int kStageWarps = 4;
constexpr int kStageTileWords = 20 * kTile / 2;  // 19 rows of 64 bytes, padded to 1280 bytes
__device__ __forceinline__ uint32_t lds_volatile_u32(const uint32_t* p) {
  return *static_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* tm, int32_t x, int32_t y,
                                       uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
#ifndef LBM_STAGES
#define LBM_STAGES 2
#endif
constexpr int kStages = LBM_STAGES;  // ring depth per warp: pairs in flight + 1
template <class S>
__global__ void __launch_bounds__(kStageWarps * 32, kStages <= 2 ? 8 : (kStages == 3 ? 6 : 5))
    k_bulk2s(const DevLattice d, const StepParams p, const __grid_constant__ CUtensorMap tm) {
  static_assert(sizeof(S) == 2, "staged rows: 16-bit storage");
  __shared__ __align__(128) uint32_t buf[kStageWarps][kStages][2][kStageTileWords];
  __shared__ __align__(8) uint64_t bars[kStageWarps][kStages];
  __shared__ __align__(16) int32_t desc_s[kStageWarps][20];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nb = d.n_boundary, n_pairs = (d.n_tiles - nb) / 2;
  const int64_t stride = (int64_t)gridDim.x * kStageWarps;
  S* P = static_cast<S*>(d.pop);
  const int64_t np = d.npad;
  if (lane == 0)
    for (int i = 0; i < kStages; ++i) mbar_init(&bars[w][i], 1);
  __syncwarp();
  // tile ids of pair qq (every lane loads the same two words)
  auto tile_of = [&](int64_t qq, int h) -> int32_t {
    return qq < n_pairs ? __ldg(&d.launch[nb + 2 * qq + h].tile) : 0;
  };
  auto issue = [&](int st, int32_t ta, int32_t tb) {
    if (lane == 0) {
      // the lanes' reads of this stage (two iterations back) come before the
      // copies that overwrite it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bars[w][st], 2u * kQ * kTile * (uint32_t)sizeof(S));
      tma_2d(&buf[w][st][0][0], &tm, ta * kTile, 0, &bars[w][st]);
      tma_2d(&buf[w][st][1][0], &tm, tb * kTile, 0, &bars[w][st]);
    }
  };
  // ring: pair q + i stride sits in stage (it + i) mod kStages; the ids of
  // a pair are loaded an iteration before its copies are issued
  int64_t q = (int64_t)blockIdx.x * kStageWarps + w;
  int32_t ta[kStages + 1], tb[kStages + 1];  // ids of pairs q, q + stride, ...
  for (int i = 0; i <= kStages; ++i) {
    ta[i] = tile_of(q + i * stride, 0);
    tb[i] = tile_of(q + i * stride, 1);
  }
  for (int i = 0; i + 1 < kStages; ++i)
    if (q + i * stride < n_pairs) issue(i, ta[i], tb[i]);
  uint32_t phases = 0;  // bit i: parity of stage i
  const F2 om = bc2(p.omega_f);
  int st = 0;
  for (; q < n_pairs; q += stride, st = st + 1 == kStages ? 0 : st + 1) {
    const int last = st == 0 ? kStages - 1 : st - 1;  // the stage read two iterations back
    if (q + (kStages - 1) * stride < n_pairs) issue(last, ta[kStages - 1], tb[kStages - 1]);
    const uint32_t ph = (phases >> st) & 1u;
    if (!__all_sync(0xFFFFFFFFu, mbar_wait_bounded(&bars[w][st], ph))) {
      // the copies did not complete: flag the step and stop (one more bounded
      // wait on each stage gives copies in flight a chance to land)
      if (lane == 0) atomicOr(d.err, kErrTimeout);
      for (int i = 0; i < kStages; ++i) mbar_wait_bounded(&bars[w][i], (phases >> i) & 1u);
      return;
    }
    phases ^= 1u << st;
    const int64_t x = (int64_t)(lane < 16 ? ta[0] : tb[0]) * kTile + 2 * (lane & 15);
    const uint32_t* row = &buf[w][st][lane >> 4][lane & 15];  // row j at + j * 16 words
    using Cd = Codec2<S>;
    collide2(
        [&](int j) -> F2 { return Cd::unpack(row[j * (kTile / 2)]); },
        [&](int j) -> F2 { return Cd::unpack(lds_volatile_u32(row + j * (kTile / 2))); }, om,
        d.err, d.err, [&](F2 s0) { Cd::st_al(P + x, s0); },
        [&](auto A, F2 sa, F2 sb) {
          constexpr int a = decltype(A)::value, b = a + 1;
          Cd::st_al(P + b * np + x, sa);
          Cd::st_al(P + a * np + x, sb);
        });
    __syncwarp();
    for (int i = 0; i < kStages; ++i) {
      ta[i] = ta[i + 1];
      tb[i] = tb[i + 1];
    }
    ta[kStages] = tile_of(q + (kStages + 1) * stride, 0);
    tb[kStages] = tile_of(q + (kStages + 1) * stride, 1);
  }
  // a lone last bulk tile
  if ((d.n_tiles - nb) % 2 && blockIdx.x == 0 && w == 0)
    bulk_tile<S, false>(d, p, d.n_tiles - 1, desc_s[w], lane);
}

template <class S, bool ODD, int W, bool DIAG = false>
__global__ void __launch_bounds__(W * 32, BulkMinBlocks<S, W>::one)
    k_bulk(const DevLattice d, const StepParams p) {
  __shared__ __align__(16) int32_t desc_s[W][20];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = d.n_boundary + (int64_t)blockIdx.x * W + w;
  if (k >= d.n_tiles) return;  // warp-uniform
  if constexpr (DIAG) bulk_tile<S, ODD, true>(d, p, k, desc_s[w], lane, d.diag_mass + k);
  else bulk_tile<S, ODD>(d, p, k, desc_s[w], lane);
}

// Resident CTAs (4 warps) per SM requested of the boundary kernel: 7, i.e. 73
// registers, measured on the long tube and the depth-6 tree against 6, 8 and
// 10 (tree FP32 +8 %, tube FP32 +3 %, FP16S +1-3 % over 8, whose 64 registers
// spill on odd steps).
#ifndef LBM_BOUNDARY_MINB
#define LBM_BOUNDARY_MINB 7
#endif
// Boundary tile at launch position k (whole warp); nbr_s, bar: the warp's
// staging area (18 rows of per-site neighbours) and mbarrier; dsc: its
// 20-word descriptor area.
// PART selects the sites updated: 0 those whose iolet links (if any) all lead
// to one iolet (boundary_fast), 1 the sites linked to two or more iolets (the
// per-link form, run by k_boundary_multi over the tiles that have such sites),
// 2 both (the persistent kernel).
template <class S, bool ODD, int PART = 0>
__device__ __forceinline__ bool boundary_tile(const DevLattice& d, const StepParams& p, int64_t k,
                                              int32_t* dsc, int32_t* nbr_s, uint64_t* bar,
                                              typename Codec<S>::C* gsm, int lane,
                                              uint32_t* bar_phase = nullptr,
                                              typename Codec<S>::C* dr = nullptr) {
  using C = typename Codec<S>::C;
  // a warp that updates tiles in a loop (persistent kernel): lanes that left
  // the previous tile early (padding sites) wait here until every lane is done
  // with its descriptor, segment table and staged rows
  __syncwarp();
  const int64_t slot = k * kTile + lane;  // boundary tiles lead the launch order
  // per-site data and the descriptor, all in one round trip
  const uint32_t smask = __ldg(d.slot_mask + slot);
  const uint32_t iom = __ldg(d.slot_io + slot);
  if (lane < 20) dsc[lane] = __ldg(reinterpret_cast<const int32_t*>(d.launch + k) + lane);
  __syncwarp();
  const uint32_t tmask = (uint32_t)dsc[18];
  const bool irr = tmask & kIrregular;
  const int64_t x = (int64_t)dsc[19] * kTile + lane;
  // odd steps of an irregular tile: its segment table (80 words, coalesced
  // loads into the staging area) when its lanes form at most kMaxSegments
  // runs of shared offsets, else its per-site neighbour rows (cp.async.bulk
  // into shared memory, completing on the warp's mbarrier); the per-link form
  // of multi-iolet sites (PART 1, 2) always reads the per-site rows
  const bool seg = ODD && irr && (tmask & kSegmented) && PART == 0;
  const bool stage = ODD && irr && !seg;
  if (seg) {
    const int32_t* src = d.seg_tab + k * kSegWords;
    for (int q = lane; q < kSegWords; q += kTile) nbr_s[q] = __ldg(src + q);
  }
  // bar_phase: a warp that stages repeatedly (persistent kernel) keeps one
  // initialised mbarrier and tracks its phase; otherwise it is set up here.
  if (stage) {
    if (lane == 0 && !bar_phase) mbar_init(bar, 1);
    __syncwarp();
    if (lane == 0) {
      // the lanes' earlier ordinary writes to the staging area (a previous
      // tile's rows turned into offsets, or its segment table) are ordered
      // before the asynchronous copies that overwrite it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, 18u * kTile * 4u);
      for (int i = 0; i < 18; ++i)
        bulk_g2s(nbr_s + i * kTile, d.slot_nbr + i * d.slot_stride + k * kTile, kTile * 4, bar);
    }
  }
  const bool valid = smask & kValid;
  // per-site wall and inlet data (F, kappa/3, inlet profile p0, ps, pc) into
  // the warp's area (from row kAreaSite), copied asynchronously so that no register
  // holds them while the populations load
  // Rows of 32 doubles: F (row 0) and p0, ps, pc (rows 2-4) in the compute
  // type at the start of their rows, kappa c_s^2 (row 1) in FP64.
  double* site = reinterpret_cast<double*>(gsm + kAreaSite * kTile);  // [5][32]
  auto site_row = [&](int r) { return reinterpret_cast<C*>(site + r * kTile); };
  if (valid && (smask & kHasWall)) {
    cp_async_elem(site_row(0) + lane, static_cast<const C*>(d.slot_F) + slot);
    cp_async8(site + kTile + lane, d.slot_kappa + slot);
  }
  if (valid && (smask & kHasInlet)) {
    const C* prof = static_cast<const C*>(d.slot_prof);
    cp_async_elem(site_row(2) + lane, prof + slot);
    cp_async_elem(site_row(3) + lane, prof + d.slot_stride + slot);
    cp_async_elem(site_row(4) + lane, prof + 2 * d.slot_stride + slot);
  }
  cp_async_commit();
  // warp-uniform: which boundary states the tile needs at all
  const bool warp_io = __any_sync(0xFFFFFFFFu, valid && (iom & kDirBits));
  const bool warp_wall = p.elastic && __any_sync(0xFFFFFFFFu, valid && (smask & kHasWall));
  const uint32_t warp_nf = __reduce_or_sync(0xFFFFFFFFu, valid ? (smask & kDirBits) : 0u);
  // sites linked to two or more iolets take the per-link form
  const bool multi = smask & kMultiIolet;
  S* P = static_cast<S*>(d.pop);
  if (stage) {
    const uint32_t ph = bar_phase ? *bar_phase : 0u;
    // one decision for the whole warp (lanes could see the limit and the
    // completion in different polls)
    if (!__all_sync(0xFFFFFFFFu, mbar_wait_bounded(bar, ph))) {
      // The copies did not complete: the step's results are invalid from here
      // on (kErrTimeout), and the caller does no further tile work with this
      // staging area.  One more bounded wait gives copies still in flight a
      // chance to land; nothing waits on them after that.
      if (lane == 0) atomicOr(d.err, kErrTimeout);
      mbar_wait_bounded(bar, ph);
      return false;
    }
    if (bar_phase) *bar_phase = ph ^ 1u;
  }
  if (seg) __syncwarp();  // the segment table is in shared memory
  if (!valid) return true;
  if (!multi) {
    if constexpr (PART != 1) {
      // this lane's offsets: the tile's (coherent tiles), its segment's, or
      // its column of the staged per-site rows turned into offsets (the rows
      // of links leaving the fluid are left as they are and never used)
      const int32_t* offp = dsc;
      int ostride = 1;
      if (seg) {
        const int q = (lane >= nbr_s[1]) + (lane >= nbr_s[2]) + (lane >= nbr_s[3]);
        offp = nbr_s + kMaxSegments + 18 * q;
      } else if (stage) {
        const uint32_t nfl = smask & kDirBits;
        for (int i = 1; i < kQ; ++i)
          if (!((nfl >> i) & 1u)) nbr_s[(i - 1) * kTile + lane] -= (int32_t)x;
        offp = nbr_s + lane;
        ostride = kTile;
      }
      const C r = boundary_fast<S, ODD>(d, p, omega_as<C>(p.omega, p.omega_f), P, x, offp,
                                        ostride, smask, iom, site, nbr_s, lane, slot, warp_io,
                                        warp_wall, warp_nf, gsm);
      if (dr) *dr = r;
    }
    return true;
  }
  if constexpr (PART == 0) return true;
  cp_async_wait_all();
  const C Fw = site_row(0)[lane];
  const double Kw = site[kTile + lane];
  const C pr0 = site_row(2)[lane], pr1 = site_row(3)[lane], pr2 = site_row(4)[lane];
  if constexpr (PART == 1) {
    C g[kQ];
    boundary_load<S, ODD>(P, d.npad, x, smask & kDirBits, dsc, irr, nbr_s, lane, g, d.n, d.err);
    const C r = boundary_update<S, ODD>(d, p, omega_as<C>(p.omega, p.omega_f), P, x, dsc, irr,
                                        smask, iom, Fw, Kw, pr0, pr1, pr2, nbr_s, lane, slot, g,
                                        gsm);
    if (dr) *dr = r;
  } else {
    boundary_slow<S, ODD>(d, p, P, x, dsc, irr, smask, iom, Fw, Kw, pr0, pr1, pr2, nbr_s, lane,
                          slot, gsm);
  }
  return true;
}

template <class S, bool ODD, bool DIAG = false>
__global__ void __launch_bounds__(kBoundaryWarps * 32, sizeof(S) == 8 ? 2 : LBM_BOUNDARY_MINB)
    k_boundary(const DevLattice d, const StepParams p0) {
  StepParams p = p0;
  p.diag = DIAG;  // a compile-time constant for the tile code
  using C = typename Codec<S>::C;
  __shared__ __align__(128) int32_t stage[kBoundaryWarps][18 * kTile];
  __shared__ __align__(16) C gs[kBoundaryWarps][BoundaryArea<C>::size];
  __shared__ __align__(16) int32_t desc_s[kBoundaryWarps][20];
  __shared__ uint64_t bars[kBoundaryWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = (int64_t)blockIdx.x * kBoundaryWarps + w;
  if (k >= d.n_boundary) return;  // warp-uniform
  C dr = C(0);
  boundary_tile<S, ODD>(d, p, k, desc_s[w], stage[w], &bars[w], gs[w], lane, nullptr, &dr);
  if constexpr (DIAG) {
    const C m = warp_sum(dr);
    if (lane == 0) d.diag_mass[k] = (double)m;
  }
}

// The sites linked to two or more iolets, over the boundary tiles that have
// such sites (d.multi_tiles); every other site of those tiles is left to
// k_boundary.
template <class S, bool ODD, bool DIAG = false>
__global__ void __launch_bounds__(kBoundaryWarps * 32)
    k_boundary_multi(const DevLattice d, const StepParams p0) {
  StepParams p = p0;
  p.diag = DIAG;
  using C = typename Codec<S>::C;
  __shared__ __align__(128) int32_t stage[kBoundaryWarps][18 * kTile];
  __shared__ __align__(16) C gs[kBoundaryWarps][BoundaryArea<C>::size];
  __shared__ __align__(16) int32_t desc_s[kBoundaryWarps][20];
  __shared__ uint64_t bars[kBoundaryWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * kBoundaryWarps + w;
  if (q >= d.n_multi) return;  // warp-uniform
  const int64_t k = __ldg(d.multi_tiles + q);
  C dr = C(0);
  boundary_tile<S, ODD, 1>(d, p, k, desc_s[w], stage[w], &bars[w], gs[w], lane, nullptr, &dr);
  if constexpr (DIAG) {
    // after k_boundary (same stream) wrote the tile's other sites
    const C m = warp_sum(dr);
    if (lane == 0) d.diag_mass[k] += (double)m;
  }
}

// -------------------------------------------------------------- ensembles
// One launch of each step kernel covers every member of an ensemble: the
// tile map names the member and launch position of each global tile (one
// 8-byte load, no search).

__device__ __forceinline__ TileRef tile_ref(const TileRef* map, int64_t g) {
  const long long v = __ldg(reinterpret_cast<const long long*>(map + g));
  return TileRef{(int32_t)(v & 0xFFFFFFFFll), (int32_t)(v >> 32)};
}

template <class S, bool ODD, int W>
__global__ void __launch_bounds__(W * 32, EnsBulkMinBlocks<S, W>::one)
    k_bulk_ens(const EnsembleLaunch e, const StepParams p) {
  __shared__ __align__(16) int32_t desc_s[W][20];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * W + w;
  if (g >= e.n_bulk_tiles) return;  // warp-uniform
  const TileRef t = tile_ref(e.bulk_map, g);
  const MemberDev& md = e.mem[t.member];
  StepParams pm = p;
  pm.omega = md.omega;
  pm.omega_f = md.omega_f;
  bulk_tile<S, ODD>(md.d, pm, t.k, desc_s[w], lane);
}

__device__ __forceinline__ BulkView member_view(const MemberDev* m) {
  const DevLattice* d = &m->d;
  BulkView v;
  v.pop = (void*)__ldg(reinterpret_cast<const unsigned long long*>(&d->pop));
  v.launch = reinterpret_cast<const LaunchDesc*>(
      __ldg(reinterpret_cast<const unsigned long long*>(&d->launch)));
  v.err = (int*)__ldg(reinterpret_cast<const unsigned long long*>(&d->err));
  v.chk = (int*)__ldg(reinterpret_cast<const unsigned long long*>(&d->chk));
  v.npad = __ldg(&d->npad);
  v.n = __ldg(&d->n);
  v.n_tiles = __ldg(&d->n_tiles);
  return v;
}

// Bulk tiles of all members, two per warp (the pair may span two members).
template <class S, bool ODD, bool VERT, int W>
__global__ void __launch_bounds__(W * 32, EnsBulkMinBlocks<S, W>::two)
    k_bulk2_ens(const EnsembleLaunch e, const StepParams p) {
  __shared__ __align__(16) int32_t desc_s[W][2][20];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g0 = 2 * ((int64_t)blockIdx.x * W + w);
  if (g0 >= e.n_bulk_tiles) return;  // warp-uniform
  const bool two = g0 + 1 < e.n_bulk_tiles;
  const TileRef ta = tile_ref(e.bulk_map, g0), tb = two ? tile_ref(e.bulk_map, g0 + 1) : ta;
  const BulkView A = member_view(e.mem + ta.member), B = member_view(e.mem + tb.member);
  bulk_pair_warp<S, ODD, VERT>(A, ta.k, __ldg(&e.mem[ta.member].omega_f), B, tb.k,
                               __ldg(&e.mem[tb.member].omega_f), two, ta.member == tb.member,
                               p.prefetch, desc_s[w], lane);
}

template <class S, bool ODD>
__global__ void __launch_bounds__(kBoundaryWarps * 32, sizeof(S) == 8 ? 2 : LBM_ENS_BOUNDARY_MINB)
    k_boundary_ens(const EnsembleLaunch e, const StepParams p) {
  using C = typename Codec<S>::C;
  __shared__ __align__(128) int32_t stage[kBoundaryWarps][18 * kTile];
  __shared__ __align__(16) C gs[kBoundaryWarps][BoundaryArea<C>::size];
  __shared__ __align__(16) int32_t desc_s[kBoundaryWarps][20];
  __shared__ uint64_t bars[kBoundaryWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t g = (int64_t)blockIdx.x * kBoundaryWarps + w;
  if (g >= e.n_boundary_tiles) return;  // warp-uniform
  const TileRef t = tile_ref(e.boundary_map, g);
  const MemberDev& md = e.mem[t.member];
  StepParams pm = p;
  pm.omega = md.omega;
  pm.omega_f = md.omega_f;
  pm.rho0 = md.rho0;
  pm.rho0_f = md.rho0_f;
  pm.rho0_exact = md.rho0_exact;
  pm.diag = 0;  // ensembles: no fused diagnostics
  pm.elastic = md.elastic;
  boundary_tile<S, ODD>(md.d, pm, t.k, desc_s[w], stage[w], &bars[w], gs[w], lane);
}

// ------------------------------------------------- persistent ensemble kernel
// Every CTA stays resident for the whole launch (cooperative launch) and
// loops over the steps: its warps take chunks of tiles from a
// per-step device counter - boundary tiles of all members first, then bulk
// tiles - and the grid meets at a barrier between steps.  The chunk grows
// with the work per warp (1 for small ensembles, where a warp's chunk is the
// critical path of a step; up to 16 for large ones, to keep the counter's
// atomics few).

constexpr int kPersistWarps = 8;
constexpr int kPersistChunkMax = 16;
constexpr long long kBarrierCycles = 1ll << 31;  // ~1 s at the GB300 SM clock

// Grid barrier: bounded spin; false (every thread of the CTA) on timeout.
__device__ bool grid_sync(GridSync* gs, unsigned expected, unsigned& gen, int next_slot, int* err) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&gs->arrive, 1u) == expected - 1u) {
      atomicExch(&gs->arrive, 0u);
      atomicExch(&gs->work[next_slot], 0ull);
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const long long t0 = clock64();
      unsigned ns = 32;
      while (*static_cast<volatile unsigned*>(&gs->gen) == gen) {
        if (clock64() - t0 > kBarrierCycles) {
          atomicOr(err, kErrTimeout);
          atomicExch(&gs->abort, 1u);
          ok = 0;
          break;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;  // short sleeps first: most waits are brief
      }
    }
    __threadfence();
    if (*static_cast<volatile unsigned*>(&gs->abort)) ok = 0;
  }
  ok = __syncthreads_and(ok);
  ++gen;
  return ok != 0;
}

// The four tile bodies as separate functions, so that each keeps the
// register allocation it has in its own kernel.
template <class S, bool ODD>
__device__ __noinline__ bool persist_boundary(const DevLattice& d, const StepParams& p, int64_t k,
                                              int32_t* dsc, int32_t* nbr_s, uint64_t* bar,
                                              typename Codec<S>::C* gsm, int lane,
                                              uint32_t* phase) {
  return boundary_tile<S, ODD, 2>(d, p, k, dsc, nbr_s, bar, gsm, lane, phase);
}
template <class S, bool ODD>
__device__ __noinline__ void persist_bulk(const DevLattice& d, const StepParams& p, int64_t k,
                                          int32_t* dsc, int lane) {
  bulk_tile<S, ODD>(d, p, k, dsc, lane);
}

template <class S>
__global__ void __launch_bounds__(kPersistWarps * 32, sizeof(S) == 8 ? 1 : 4)
    k_ensemble_persistent(const EnsembleLaunch e, const StepParams p, int64_t n_steps,
                          GridSync* gs, unsigned expected, int chunk) {
  using C = typename Codec<S>::C;
  __shared__ __align__(128) int32_t stage[kPersistWarps][18 * kTile];
  __shared__ __align__(16) C gsm[kPersistWarps][BoundaryArea<C>::size];
  __shared__ __align__(16) int32_t desc_s[kPersistWarps][20];
  __shared__ uint64_t bars[kPersistWarps];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) mbar_init(&bars[w], 1);
  __syncwarp();
  uint32_t phase = 0;
  unsigned gen = 0;  // the launcher clears the barrier state
  int* err0 = e.mem[0].d.err;
  const int64_t total = e.n_boundary_tiles + e.n_bulk_tiles;
  for (int64_t s = 0; s < n_steps; ++s) {
    StepParams q = p;
    q.step = p.step + s;
    q.write_state = s == n_steps - 1 ? 1 : 0;
    const bool odd = q.step & 1;
    const int slot = (int)(q.step & 1);
    bool stop = false;  // this warp's staging timed out: no further tile work
    for (;;) {
      unsigned long long t0 = 0;
      if (lane == 0) {
        t0 = *static_cast<volatile unsigned*>(&gs->abort) ? (unsigned long long)total
                                                          : atomicAdd(&gs->work[slot],
                                                                      (unsigned long long)chunk);
      }
      t0 = __shfl_sync(0xffffffffu, t0, 0);
      if ((int64_t)t0 >= total) break;
      const int64_t t1 = (int64_t)t0 + chunk < total ? (int64_t)t0 + chunk : total;
      for (int64_t t = (int64_t)t0; t < t1; ++t) {
        if (t < e.n_boundary_tiles) {
          const TileRef tr = tile_ref(e.boundary_map, t);
          const MemberDev& md = e.mem[tr.member];
          StepParams pm = q;
          pm.omega = md.omega;
          pm.omega_f = md.omega_f;
          pm.rho0 = md.rho0;
          pm.rho0_f = md.rho0_f;
          pm.rho0_exact = md.rho0_exact;
          pm.diag = 0;  // ensembles: no fused diagnostics
          pm.elastic = md.elastic;
          const int64_t k = tr.k;
          const bool ok = odd ? persist_boundary<S, true>(md.d, pm, k, desc_s[w], stage[w],
                                                          &bars[w], gsm[w], lane, &phase)
                              : persist_boundary<S, false>(md.d, pm, k, desc_s[w], stage[w],
                                                           &bars[w], gsm[w], lane, &phase);
          if (!ok) {
            if (lane == 0) atomicExch(&gs->abort, 1u);
            stop = true;
            break;
          }
        } else {
          const TileRef tr = tile_ref(e.bulk_map, t - e.n_boundary_tiles);
          const MemberDev& md = e.mem[tr.member];
          StepParams pm = q;
          pm.omega = md.omega;
          pm.omega_f = md.omega_f;
          const int64_t k = tr.k;
          if (odd) persist_bulk<S, true>(md.d, pm, k, desc_s[w], lane);
          else persist_bulk<S, false>(md.d, pm, k, desc_s[w], lane);
        }
        __syncwarp();
      }
      if (stop) break;
    }
    if (!grid_sync(gs, expected, gen, slot ^ 1, err0)) return;
  }
}

template <class S>
int ensemble_persistent_t(const EnsembleLaunch& e, const StepParams& p, int64_t n_steps,
                          GridSync* gs, int extra, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t r = cudaGetDevice(&dev);
  if (r == cudaSuccess) r = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (r == cudaSuccess)
    r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ensemble_persistent<S>,
                                                      kPersistWarps * 32, 0);
  if (r != cudaSuccess) return (int)r;
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  const unsigned blocks = (unsigned)(per_sm * sms);
  r = cudaMemsetAsync(gs, 0, sizeof(GridSync), s);
  if (r != cudaSuccess) return (int)r;
  unsigned expected = blocks + (unsigned)(extra > 0 ? extra : 0);
  const int64_t per_warp = (e.n_boundary_tiles + e.n_bulk_tiles) / ((int64_t)blocks * kPersistWarps * 8);
  int chunk = (int)(per_warp < 1 ? 1 : (per_warp > kPersistChunkMax ? kPersistChunkMax : per_warp));
  void* args[] = {(void*)&e, (void*)&p, (void*)&n_steps, (void*)&gs, (void*)&expected, (void*)&chunk};
  r = cudaLaunchCooperativeKernel((const void*)k_ensemble_persistent<S>, dim3(blocks),
                                  dim3(kPersistWarps * 32), args, 0, s);
  return (int)r;
}

__global__ void k_advance(int64_t* step, int64_t by) { *step += by; }
__global__ void k_set_step(int64_t* step, int64_t value) { *step = value; }

// ------------------------------------------------ state conversion kernels

// Fluid neighbours and non-fluid mask of site x from the tile tables.
__device__ void site_links(const DevLattice& d, int64_t x, uint32_t& nf, int64_t (&nb)[kQ]) {
  const TileDesc& td = d.tiles[x >> 5];
  nb[0] = x;
  if (td.mask == 0) {
    nf = 0;
    for (int i = 1; i < kQ; ++i) nb[i] = x + td.code[i - 1];
    return;
  }
  const int64_t slot = (int64_t)td.slot + (x & 31);
  nf = d.slot_mask[slot] & kDirBits;
  const bool irr = td.mask & kIrregular;
  for (int i = 1; i < kQ; ++i)
    nb[i] = irr ? (int64_t)d.slot_nbr[(i - 1) * d.slot_stride + slot] : x + td.code[i - 1];
}

// Storage index holding the pre-collision population j of site x.
__device__ __forceinline__ int64_t slot_of(const DevLattice& d, int64_t x, int j, bool odd,
                                           uint32_t nf, const int64_t (&nb)[kQ]) {
  if (!odd || j == 0) return j * d.npad + x;
  const int o = dir_opp(j);
  if ((nf >> o) & 1u) return j * d.npad + x;
  return o * d.npad + nb[o];
}

// f = f^eq(rho, u) (Eq. feq) at every site, stored as g^eq = f^eq - w in
// the compute type (FP64 storage: FP64; else FP32, which the FP32 collision
// would round to anyway, and no FP64 arithmetic on the slow FP64 pipe).
template <class S>
__global__ void k_init(const DevLattice d, const double* rho, const double* u) {
  using C = typename Codec<S>::C;
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n) return;
  const double r = rho ? rho[x] : 1.0;
  const C dr = C(r - 1.0), rc = C(r);
  const C ux = u ? C(u[3 * x]) : C(0), uy = u ? C(u[3 * x + 1]) : C(0);
  const C uz = u ? C(u[3 * x + 2]) : C(0);
  const C usq = C(1.5) * (ux * ux + uy * uy + uz * uz);
  S* P = static_cast<S*>(d.pop);
  unroll<kQ>([&](auto I) {
    constexpr int i = decltype(I)::value;
    Codec<S>::st(P + i * d.npad + x, i, geq<i, C>(dr, rc, ux, uy, uz, usq));
  });
}

template <class S>
__global__ void k_gather(const DevLattice d, int odd, double* f) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n) return;
  uint32_t nf;
  int64_t nb[kQ];
  site_links(d, x, nf, nb);
  const S* P = static_cast<const S*>(d.pop);
  for (int j = 0; j < kQ; ++j) f[kQ * x + j] = Codec<S>::get(P + slot_of(d, x, j, odd, nf, nb), j);
}

template <class S>
__global__ void k_scatter(const DevLattice d, int odd, const double* f) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n) return;
  uint32_t nf;
  int64_t nb[kQ];
  site_links(d, x, nf, nb);
  S* P = static_cast<S*>(d.pop);
  for (int j = 0; j < kQ; ++j) Codec<S>::put(P + slot_of(d, x, j, odd, nf, nb), j, f[kQ * x + j]);
}

template <class S>
__device__ void site_f(const DevLattice& d, int64_t x, bool odd, double (&f)[kQ]) {
  uint32_t nf;
  int64_t nb[kQ];
  site_links(d, x, nf, nb);
  const S* P = static_cast<const S*>(d.pop);
  for (int j = 0; j < kQ; ++j) f[j] = Codec<S>::get(P + slot_of(d, x, j, odd, nf, nb), j);
}

__device__ void f_moments(const double (&f)[kQ], double& rho, double& jx, double& jy, double& jz) {
  rho = 0.0; jx = 0.0; jy = 0.0; jz = 0.0;
  for (int j = 0; j < kQ; ++j) {
    rho += f[j];
    jx += f[j] * dir_x(j);
    jy += f[j] * dir_y(j);
    jz += f[j] * dir_z(j);
  }
}

// rho, u of every site (Eqs. Density, Momentum), canonical order.  FP64
// storage: in FP64 from f; the other storages: from the stored g in the
// compute type, as the step kernels form them (rho = 1 + sum g in FP64).
template <class S>
__global__ void k_moments(const DevLattice d, int odd, double* rho, double* u) {
  using C = typename Codec<S>::C;
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= d.n) return;
  if constexpr (std::is_same<C, double>::value) {
    double f[kQ], r, jx, jy, jz;
    site_f<S>(d, x, odd, f);
    f_moments(f, r, jx, jy, jz);
    if (rho) rho[x] = r;
    if (u) {
      u[3 * x] = jx / r;
      u[3 * x + 1] = jy / r;
      u[3 * x + 2] = jz / r;
    }
  } else {
    uint32_t nf;
    int64_t nb[kQ];
    site_links(d, x, nf, nb);
    const S* P = static_cast<const S*>(d.pop);
    C g[kQ];
    for (int j = 0; j < kQ; ++j) g[j] = Codec<S>::ld(P + slot_of(d, x, j, odd, nf, nb), j);
    const Mom<C> m = moments(g);
    if (rho) rho[x] = 1.0 + (double)m.drho;
    if (u) {
      u[3 * x] = m.ux;
      u[3 * x + 1] = m.uy;
      u[3 * x + 2] = m.uz;
    }
  }
}

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;                        // partials of one reduction
constexpr int kMassBlocks = 768;                        // partials [0, 768): mass
constexpr int kFluxPartials = kRedBlocks - kMassBlocks;  // [768, 1024): iolet fluxes
constexpr int kFluxBlocksMax = 16;                      // blocks per iolet

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// Checked builds: every slot of a valid site stored exactly once since the
// last check, padding slots never; the counts are cleared for the next step.
__global__ void k_check_counts(int* chk, int64_t total, int64_t npad, int64_t n, int* err) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int want = (q % npad) < n ? 1 : 0;
    if (chk[q] != want) atomicOr(err, kErrCheck);
    chk[q] = 0;
  }
}

// Mass partials: fixed grid, fixed order -> deterministic.  Both AA layouts
// hold every population of every site exactly once (each step writes every
// slot once), so the total mass is n + the sum of all stored g = f - w, read
// as a flat stream: no neighbour gather and no momentum.  Each site's 19
// values are summed in the compute type (exact data for every storage, FP32
// adds of |g| << 1 for the FP32 paths) and the sites in FP64.
template <class S>
__global__ void __launch_bounds__(kRedThreads) k_mass(const DevLattice d, double* partial) {
  using Cd = Codec<S>;
  using C = typename Cd::C;
  __shared__ double sh[kRedThreads];
  const S* P = static_cast<const S*>(d.pop);
  double acc = 0.0;
  for (int64_t x = (int64_t)blockIdx.x * kRedThreads + threadIdx.x; x < d.n;
       x += (int64_t)kMassBlocks * kRedThreads) {
    C sg = C(0);
    unroll<kQ>([&](auto J) {
      constexpr int j = decltype(J)::value;
      sg += Cd::ld(P + j * d.npad + x, j);
    });
    acc += (double)sg;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads) k_mass_final(const double* partial, int64_t n,
                                                            int* err, double* out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int b = threadIdx.x; b < kMassBlocks; b += kRedThreads) acc += partial[b];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    out[0] = (double)n + s;
    if (!isfinite(s)) atomicOr(err, kErrUnstable);  // a non-finite population anywhere
  }
}

// Flux of rho u along iolet k's axis over the sites touching it: blocks
// (k, b) of a (n_iolets x bpi) grid take every bpi-th chunk of the site list;
// with bpi > 1 they write partials that k_flux_final adds in block order,
// with bpi = 1 the single block writes the result.
template <class S>
__global__ void __launch_bounds__(kRedThreads)
    k_flux(const DevLattice d, int odd, const int64_t* off, const int64_t* sites, double* part,
           double* out) {
  __shared__ double sh[kRedThreads];
  const int k = blockIdx.x, b = blockIdx.y, bpi = gridDim.y;
  const IoletDev& io = d.iolets[k];
  double acc = 0.0;
  for (int64_t q = off[k] + (int64_t)b * kRedThreads + threadIdx.x; q < off[k + 1];
       q += (int64_t)bpi * kRedThreads) {
    double f[kQ], r, jx, jy, jz;
    site_f<S>(d, sites[q], odd, f);
    f_moments(f, r, jx, jy, jz);
    acc += jx * io.axis[0] + jy * io.axis[1] + jz * io.axis[2];
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    if (bpi == 1) out[1 + k] = s;
    else part[k * bpi + b] = s;
  }
}

// Fused diagnostics, the final sums in a fixed order.  Blocks [0, kDiagBlocks)
// add contiguous ranges of the per-tile partials of rho - 1; then fpi blocks
// per iolet k add (rho u) . axis_k over consecutive runs of kRedThreads of its
// sites (io_q: their places in diag_j; one site per thread, so no block waits
// on a chain of dependent loads).  Every block writes one partial; the last
// block to finish adds them in block order: out[0] = n + the mass partials,
// out[1 + k] = iolet k's fpi partials.
constexpr int kDiagBlocks = 128;
__global__ void __launch_bounds__(kRedThreads)
    k_diag_final(const DevLattice d, const int64_t* io_off, const int64_t* io_q, int fpi,
                 double* part, unsigned* done, double* out) {
  __shared__ double sh[kRedThreads];
  __shared__ int last;
  const int b = blockIdx.x;
  double acc = 0.0;
  if (b < kDiagBlocks) {
    const int64_t per = (d.n_tiles + kDiagBlocks - 1) / kDiagBlocks;
    const int64_t lo = (int64_t)b * per;
    const int64_t hi = lo + per < d.n_tiles ? lo + per : d.n_tiles;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) acc += d.diag_mass[i];
  } else {
    const int k = (b - kDiagBlocks) / fpi, f = (b - kDiagBlocks) % fpi;
    const int64_t q = io_off[k] + (int64_t)f * kRedThreads + threadIdx.x;
    if (q < io_off[k + 1]) {
      const IoletDev& io = d.iolets[k];
      const int64_t js = d.diag_jstride, j = io_q[q];
      acc = d.diag_j[j] * io.axis[0] + d.diag_j[js + j] * io.axis[1] +
            d.diag_j[2 * js + j] * io.axis[2];
    }
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    part[b] = s;
    __threadfence();
    last = atomicAdd(done, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;  // block-uniform
  __threadfence();
  // mass: the kDiagBlocks partials in block order
  double a = 0.0;
  for (int i = threadIdx.x; i < kDiagBlocks; i += kRedThreads) a += __ldcg(part + i);
  const double t = block_sum(a, sh);
  if (threadIdx.x == 0) {
    out[0] = (double)d.n + t;
    if (!isfinite(t)) atomicOr(d.err, kErrUnstable);
    *done = 0;  // for the next diagnostic step (stream order)
  }
  // fluxes: one warp per iolet at a time, its fpi partials in order
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = w; k < d.n_iolets; k += kRedThreads / 32) {
    const double* pk = part + kDiagBlocks + (int64_t)k * fpi;
    double v = 0.0;
    for (int f = lane; f < fpi; f += 32) v += __ldcg(pk + f);
    v = warp_sum(v);
    if (lane == 0) out[1 + k] = v;
  }
}

__global__ void k_flux_final(const double* part, int bpi, double* out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < bpi; ++b) s += part[blockIdx.x * bpi + b];
  out[1 + blockIdx.x] = s;
}

// Wall shear stress (metric): sigma = -(1 - 1/(2 tau)) sum f^neq c c,
// t = sigma n, WSS = |t - (t.n) n|.
template <class S>
__global__ void k_wss(const DevLattice d, int odd, double tau, const int64_t* sites,
                      const double* normals, int64_t m, double* out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= m) return;
  double f[kQ], r, jx, jy, jz;
  site_f<S>(d, sites[q], odd, f);
  f_moments(f, r, jx, jy, jz);
  const double ux = jx / r, uy = jy / r, uz = jz / r;
  const double usq = 1.5 * (ux * ux + uy * uy + uz * uz);
  double Pm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  unroll<kQ>([&](auto I) {
    constexpr int i = decltype(I)::value;
    const double fe = weight<double>(i) + geq<i, double>(r - 1.0, r, ux, uy, uz, usq);
    const double fn = f[i] - fe;
    const int c[3] = {dir_x(i), dir_y(i), dir_z(i)};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Pm[a][b] += fn * c[a] * c[b];
  });
  const double* n = normals + 3 * q;
  const double k = -(1.0 - 0.5 / tau);
  double t[3], tn = 0.0;
  for (int a = 0; a < 3; ++a) t[a] = k * (Pm[a][0] * n[0] + Pm[a][1] * n[1] + Pm[a][2] * n[2]);
  for (int a = 0; a < 3; ++a) tn += t[a] * n[a];
  double s2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double ta = t[a] - tn * n[a];
    s2 += ta * ta;
  }
  out[q] = sqrt(s2);
}

// ------------------------------------------------------------- dispatch

// The multi-iolet sites of one lattice (nothing when it has none).
template <class S>
void launch_multi(const DevLattice& d, const StepParams& p, bool odd, cudaStream_t s) {
  if (d.n_multi <= 0) return;
  const unsigned nb = (unsigned)((d.n_multi + kBoundaryWarps - 1) / kBoundaryWarps);
  if (p.diag) {
    if (odd) k_boundary_multi<S, true, true><<<nb, kBoundaryWarps * 32, 0, s>>>(d, p);
    else k_boundary_multi<S, false, true><<<nb, kBoundaryWarps * 32, 0, s>>>(d, p);
  } else {
    if (odd) k_boundary_multi<S, true><<<nb, kBoundaryWarps * 32, 0, s>>>(d, p);
    else k_boundary_multi<S, false><<<nb, kBoundaryWarps * 32, 0, s>>>(d, p);
  }
}

// Pairing of the bulk kernel's two sites per lane for this step's parity
// (LBM_TUNE_BULK_SITES): 0 one site per lane, 1 z-adjacent sites of one tile
// (packed words), 2 the same lane of two tiles (scalar, aligned).
inline int bulk_pairing(int32_t bulk_sites, bool odd) {
  switch (bulk_sites) {
    case 2: return odd ? 2 : 1;
    case 3: return 1;
    case 4: return 2;
    case 5: return odd ? 2 : 3;  // 3: staged rows (k_bulk2s, 16-bit even steps)
  }
  return 0;
}

// The bulk kernel of one step with W warps per CTA (pairing: bulk_pairing).
template <class S, int W, bool DIAG = false>
void launch_bulk(const DevLattice& d, const StepParams& p, bool odd, int pairing, int64_t tiles,
                 cudaStream_t m) {
  if constexpr (sizeof(S) == 2 && !DIAG) {
    if (pairing == 3 && !odd && p.n_sms > 0) {
      const int64_t pairs = tiles / 2;
      int64_t g = (int64_t)p.n_sms * (kStages <= 2 ? 8 : (kStages == 3 ? 6 : 5));
      const int64_t gmax = (pairs + kStageWarps - 1) / kStageWarps;
      if (g > gmax) g = gmax > 0 ? gmax : 1;
      if (p.tmap) {
        k_bulk2s<S><<<(unsigned)g, kStageWarps * 32, 0, m>>>(
            d, p, *static_cast<const CUtensorMap*>(p.tmap));
        return;
      }
    }
  }
  if (pairing == 3) pairing = 1;  // other storages and diagnostic steps: adjacent pairs
  if (pairing) {
    const unsigned nb = (unsigned)((tiles + 2 * W - 1) / (2 * W));
    if constexpr (sizeof(S) < 8) {
      if (pairing == 1) {
        if (odd) k_bulk2<S, true, false, W, DIAG><<<nb, W * 32, 0, m>>>(d, p);
        else k_bulk2<S, false, false, W, DIAG><<<nb, W * 32, 0, m>>>(d, p);
      } else {
        if (odd) k_bulk2<S, true, true, W, DIAG><<<nb, W * 32, 0, m>>>(d, p);
        else k_bulk2<S, false, true, W, DIAG><<<nb, W * 32, 0, m>>>(d, p);
      }
    }
  } else {
    const unsigned nb = (unsigned)((tiles + W - 1) / W);
    if (odd) k_bulk<S, true, W, DIAG><<<nb, W * 32, 0, m>>>(d, p);
    else k_bulk<S, false, W, DIAG><<<nb, W * 32, 0, m>>>(d, p);
  }
}
template <class S, int W>
void launch_bulk_ens(const EnsembleLaunch& e, const StepParams& p, bool odd, int pairing,
                     cudaStream_t m) {
  if (pairing == 3) pairing = 1;  // staged rows: single lattices only
  if (pairing) {
    const unsigned nb = (unsigned)((e.n_bulk_tiles + 2 * W - 1) / (2 * W));
    if constexpr (sizeof(S) < 8) {
      if (pairing == 1) {
        if (odd) k_bulk2_ens<S, true, false, W><<<nb, W * 32, 0, m>>>(e, p);
        else k_bulk2_ens<S, false, false, W><<<nb, W * 32, 0, m>>>(e, p);
      } else {
        if (odd) k_bulk2_ens<S, true, true, W><<<nb, W * 32, 0, m>>>(e, p);
        else k_bulk2_ens<S, false, true, W><<<nb, W * 32, 0, m>>>(e, p);
      }
    }
  } else {
    const unsigned nb = (unsigned)((e.n_bulk_tiles + W - 1) / W);
    if (odd) k_bulk_ens<S, true, W><<<nb, W * 32, 0, m>>>(e, p);
    else k_bulk_ens<S, false, W><<<nb, W * 32, 0, m>>>(e, p);
  }
}

// One step: k_boundary on the side stream, k_bulk on the main stream, joined
// on the main stream.  ev (profiling): before the fork, after k_bulk, after
// the join, all on the main stream.
template <class S>
int step_t(const DevLattice& d, const StepParams& p, const StepStreams& ss, void* const* ev) {
  cudaStream_t m = (cudaStream_t)ss.main, side = (cudaStream_t)ss.side;

  const unsigned nbnd = (unsigned)((d.n_boundary + kBoundaryWarps - 1) / kBoundaryWarps);
  const int64_t nbulk_tiles = d.n_tiles - d.n_boundary;
  const bool odd = p.step & 1;
  if (ev) cudaEventRecord((cudaEvent_t)ev[0], m);
  if (nbnd) {
    cudaEventRecord((cudaEvent_t)ss.fork, m);
    cudaStreamWaitEvent(side, (cudaEvent_t)ss.fork, 0);
    if (p.diag) {
      if (odd) k_boundary<S, true, true><<<nbnd, kBoundaryWarps * 32, 0, side>>>(d, p);
      else k_boundary<S, false, true><<<nbnd, kBoundaryWarps * 32, 0, side>>>(d, p);
    } else {
      if (odd) k_boundary<S, true><<<nbnd, kBoundaryWarps * 32, 0, side>>>(d, p);
      else k_boundary<S, false><<<nbnd, kBoundaryWarps * 32, 0, side>>>(d, p);
    }
    launch_multi<S>(d, p, odd, side);
  }
  if (nbulk_tiles > 0) {
    const int pairing = sizeof(S) < 8 ? bulk_pairing(p.bulk_sites, odd) : 0;
    // diagnostic steps take CTAs of 4 warps whatever the knob (same results)
    if (p.diag) launch_bulk<S, 4, true>(d, p, odd, pairing, nbulk_tiles, m);
    else if (p.bulk_warps == 8) launch_bulk<S, 8>(d, p, odd, pairing, nbulk_tiles, m);
    else launch_bulk<S, 4>(d, p, odd, pairing, nbulk_tiles, m);
  }
  if (ev) cudaEventRecord((cudaEvent_t)ev[1], m);
  if (nbnd) {
    cudaEventRecord((cudaEvent_t)ss.join, side);
    cudaStreamWaitEvent(m, (cudaEvent_t)ss.join, 0);
  }
  if (ev) cudaEventRecord((cudaEvent_t)ev[2], m);
  return (int)cudaGetLastError();
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <class F>
int dispatch(int storage, F&& f) {
  switch (storage) {
    case LBM_F64: return f((double*)nullptr);
    case LBM_F32: return f((float*)nullptr);
    case LBM_F16S: return f((__half*)nullptr);
    case LBM_BF16S: return f((__nv_bfloat16*)nullptr);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace

size_t storage_bytes(int storage) {
  switch (storage) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    default: return 2;
  }
}

int reduce_partials() { return kRedBlocks; }

int launch_step(int storage, const DevLattice& d, const StepParams& p, const StepStreams& ss,
                void* const* events) {
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    return step_t<S>(d, p, ss, events);
  });
}

template <class S>
int ensemble_step_t(const EnsembleLaunch& e, const StepParams& p, const StepStreams& ss) {
  cudaStream_t m = (cudaStream_t)ss.main, side = (cudaStream_t)ss.side;
  const unsigned nbnd = (unsigned)((e.n_boundary_tiles + kBoundaryWarps - 1) / kBoundaryWarps);
  const bool odd = p.step & 1;  // every member is at the same step; graphs keep the parity
  if (nbnd) {
    cudaEventRecord((cudaEvent_t)ss.fork, m);
    cudaStreamWaitEvent(side, (cudaEvent_t)ss.fork, 0);
    if (odd) k_boundary_ens<S, true><<<nbnd, kBoundaryWarps * 32, 0, side>>>(e, p);
    else k_boundary_ens<S, false><<<nbnd, kBoundaryWarps * 32, 0, side>>>(e, p);
    for (int32_t q = 0; q < e.n_multi_members; ++q) {
      const MemberDev& md = e.multi_host[q];
      StepParams pm = p;
      pm.omega = md.omega;
      pm.omega_f = md.omega_f;
      pm.rho0 = md.rho0;
      pm.rho0_f = md.rho0_f;
      pm.rho0_exact = md.rho0_exact;
      pm.diag = 0;  // ensembles: no fused diagnostics
      pm.elastic = md.elastic;
      launch_multi<S>(md.d, pm, odd, side);
    }
  }
  if (e.n_bulk_tiles > 0) {
    const int pairing = sizeof(S) < 8 ? bulk_pairing(p.bulk_sites, odd) : 0;
    if (p.bulk_warps == 8) launch_bulk_ens<S, 8>(e, p, odd, pairing, m);
    else launch_bulk_ens<S, 4>(e, p, odd, pairing, m);
  }
  if (nbnd) {
    cudaEventRecord((cudaEvent_t)ss.join, side);
    cudaStreamWaitEvent(m, (cudaEvent_t)ss.join, 0);
  }
  return (int)cudaGetLastError();
}

int launch_ensemble_step(int storage, const EnsembleLaunch& e, const StepParams& p,
                         const StepStreams& ss) {
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    return ensemble_step_t<S>(e, p, ss);
  });
}

int launch_ensemble_persistent(int storage, const EnsembleLaunch& e, const StepParams& p,
                               int64_t n_steps, GridSync* gs, int extra_arrivals, void* stream) {
  if (n_steps <= 0) return 0;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    return ensemble_persistent_t<S>(e, p, n_steps, gs, extra_arrivals, (cudaStream_t)stream);
  });
}

int launch_set_step(int64_t* step_dev, int64_t value, void* stream) {
  k_set_step<<<1, 1, 0, (cudaStream_t)stream>>>(step_dev, value);
  return (int)cudaGetLastError();
}
int launch_advance(int64_t* step_dev, int64_t by, void* stream) {
  k_advance<<<1, 1, 0, (cudaStream_t)stream>>>(step_dev, by);
  return (int)cudaGetLastError();
}

int launch_check_counts(const DevLattice& d, void* stream) {
  if (!d.chk) return 0;
  const int64_t total = (int64_t)kQ * d.npad;
  k_check_counts<<<blocks_for(total, 256) < 4096 ? blocks_for(total, 256) : 4096, 256, 0,
                   (cudaStream_t)stream>>>(d.chk, total, d.npad, d.n, d.err);
  return (int)cudaGetLastError();
}

int launch_init(int storage, const DevLattice& d, const double* rho, const double* u,
                void* stream) {
  if (d.n == 0) return 0;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_init<S><<<blocks_for(d.n, 256), 256, 0, (cudaStream_t)stream>>>(d, rho, u);
    return (int)cudaGetLastError();
  });
}

int launch_gather(int storage, const DevLattice& d, int odd, double* f, void* stream) {
  if (d.n == 0) return 0;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_gather<S><<<blocks_for(d.n, 128), 128, 0, (cudaStream_t)stream>>>(d, odd, f);
    return (int)cudaGetLastError();
  });
}

int launch_scatter(int storage, const DevLattice& d, int odd, const double* f, void* stream) {
  if (d.n == 0) return 0;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_scatter<S><<<blocks_for(d.n, 128), 128, 0, (cudaStream_t)stream>>>(d, odd, f);
    return (int)cudaGetLastError();
  });
}

int launch_moments(int storage, const DevLattice& d, int odd, double* rho, double* u,
                   void* stream) {
  if (d.n == 0) return 0;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_moments<S><<<blocks_for(d.n, 128), 128, 0, (cudaStream_t)stream>>>(d, odd, rho, u);
    return (int)cudaGetLastError();
  });
}

int launch_reduce(int storage, const DevLattice& d, int odd, const int64_t* off,
                  const int64_t* sites, double* partial, int n_partial, double* out,
                  void* stream) {
  if (n_partial < kRedBlocks) return (int)cudaErrorInvalidValue;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    cudaStream_t s = (cudaStream_t)stream;
    k_mass<S><<<kMassBlocks, kRedThreads, 0, s>>>(d, partial);
    k_mass_final<<<1, kRedThreads, 0, s>>>(partial, d.n, d.err, out);
    if (d.n_iolets > 0) {
      int bpi = kFluxPartials / d.n_iolets;
      bpi = bpi < 1 ? 1 : (bpi > kFluxBlocksMax ? kFluxBlocksMax : bpi);
      double* part = partial + kMassBlocks;
      k_flux<S><<<dim3(d.n_iolets, bpi), kRedThreads, 0, s>>>(d, odd, off, sites, part, out);
      if (bpi > 1) k_flux_final<<<d.n_iolets, 32, 0, s>>>(part, bpi, out);
    }
    return (int)cudaGetLastError();
  });
}

int launch_diag_final(const DevLattice& d, const int64_t* io_off, const int64_t* io_q, int fpi,
                      double* part, unsigned* done, double* out, void* stream) {
  k_diag_final<<<kDiagBlocks + d.n_iolets * fpi, kRedThreads, 0, (cudaStream_t)stream>>>(
      d, io_off, io_q, fpi, part, done, out);
  return (int)cudaGetLastError();
}
int diag_blocks(int n_iolets, int fpi) { return kDiagBlocks + n_iolets * fpi; }
int diag_flux_blocks(int64_t max_sites) {
  const int64_t f = (max_sites + kRedThreads - 1) / kRedThreads;
  return f > 0 ? (int)f : 1;
}

int launch_wss(int storage, const DevLattice& d, int odd, double tau, const int64_t* sites,
               const double* normals, int64_t m, double* out, void* stream) {
  if (m == 0) return 0;
  return dispatch(storage, [&](auto tag) {
    using S = std::remove_pointer_t<decltype(tag)>;
    k_wss<S><<<blocks_for(m, 128), 128, 0, (cudaStream_t)stream>>>(d, odd, tau, sites, normals,
                                                                    m, out);
    return (int)cudaGetLastError();
  });
}

}  // namespace lbm
