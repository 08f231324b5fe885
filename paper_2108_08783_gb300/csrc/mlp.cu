// Learned warm start (include/lbm_mlp.h): the network's forward pass,
// loss, back-propagation and Adam step, and the per-site feature / field
// kernels that connect it to a lattice.  No counterpart in the paper.
//
// Every contraction (forward z = h W^T, input error d W, weight gradient
// d^T h) runs through one GEMM kernel on the fifth-generation tensor cores:
// bfloat16 operands staged in shared memory in the canonical K-major layout,
// tcgen05.mma (kind::f16, 128 x 128 x 16) accumulating in FP32 in tensor
// memory, completion tracked by an mbarrier (bounded wait), and a fused
// epilogue read back with tcgen05.ld (bias + tanh + bfloat16 store; bias +
// FP32 store; tanh derivative + bfloat16 store; FP32 atomic accumulation for
// split-batch weight gradients).  The network is narrow (a few hundred
// columns), so the operands live in L2 and a GEMM launch lasts microseconds.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"

namespace {

using bf16 = __nv_bfloat16;

// ------------------------------------------------------------------ GEMM
// C(m, n) = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn]; blockIdx.z takes rows k in [z kchunk, (z+1) kchunk).
struct GemmArgs {
  const bf16* A;
  int64_t sam, sak;
  const bf16* B;
  int64_t sbk, sbn;
  int64_t M, N, K, kchunk;
  const float* bias;   // [N]            (kEpiTanh, kEpiLinear)
  const bf16* hprev;   // [M][ldh]       (kEpiDTanh)
  int64_t ldh;
  bf16* o16;           // [M][ldo]       (kEpiTanh, kEpiDTanh)
  float* o32;          // [M][ldo]       (kEpiLinear, kEpiAccum)
  int64_t ldo;
  int* err;            // set if a bounded wait for the tensor cores gives up
};

enum { kEpiTanh = 0, kEpiLinear = 1, kEpiDTanh = 2, kEpiAccum = 3 };

// Tile of one CTA: a 128 x 128 block of C, K staged 64 at a time; the UMMA
// shape is M = 128, N = 128, K = 16 (kind::f16, bf16 in, FP32 accumulate).
constexpr int kTM = 128, kTN = 128, kTK = 64, kTcThreads = 128;
constexpr uint32_t kTmemCols = 128;  // FP32 accumulator columns (= kTN)
constexpr int kTcSmemPad = 15 * 1024;

// Shared-memory tiles in the canonical K-major layout without swizzling: a
// core matrix is 8 rows x 16 bytes (8 bf16 along K) stored contiguously;
// core matrices adjacent along K are kLBO bytes apart, 8-row groups kSBO.
constexpr uint32_t kLBO = 128, kSBO = (kTK / 8) * 128;

__device__ __forceinline__ int canon(int r, int k) {  // bf16 index of element (r, k)
  return (r >> 3) * (int)(kSBO / 2) + (k >> 3) * (int)(kLBO / 2) + (r & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets, each >> 4; bits 46-48 = 0b001; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(kLBO >> 4) << 16) |
         ((uint64_t)(kSBO >> 4) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

__device__ __forceinline__ void mbar_init1(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: each try_wait suspends for a hardware-chosen interval, so the
// limit is reached only if the tensor-core work never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}

// Stage rows [row0, row0 + rows) x k [k0, k0 + kTK) of an operand whose
// element (row, k) is src[row s_row + k s_k] into T in the canonical layout,
// zero outside row < row_lim, k < ke.  16-byte loads when the operand is
// contiguous along k (one core-matrix row per load) or along rows (8 rows of
// one k per load), else element by element.
__device__ __forceinline__ void stage_tile(bf16* T, const bf16* src, int64_t s_row, int64_t s_k,
                                           int64_t row0, int64_t row_lim, int64_t k0, int64_t ke,
                                           int rows, int tid) {
  const bf16 zero = __float2bfloat16_rn(0.0f);
  const bool al = ((uintptr_t)src & 15u) == 0;
  if (al && s_k == 1 && (s_row & 7) == 0) {
    for (int e = tid; e < rows * (kTK / 8); e += kTcThreads) {
      const int r = e / (kTK / 8), c = (e % (kTK / 8)) * 8;
      const int64_t row = row0 + r, k = k0 + c;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (row < row_lim) {
        const bf16* p = src + row * s_row + k;
        if (k + 8 <= ke) {
          v = __ldg(reinterpret_cast<const uint4*>(p));
        } else {
          bf16 t[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) t[i] = (k + i < ke) ? p[i] : zero;
          v = *reinterpret_cast<const uint4*>(t);
        }
      }
      *reinterpret_cast<uint4*>(T + canon(r, c)) = v;
    }
  } else if (al && s_row == 1 && (s_k & 7) == 0 && (rows & 7) == 0) {
    for (int e = tid; e < (rows / 8) * kTK; e += kTcThreads) {
      const int r = (e % (rows / 8)) * 8, c = e / (rows / 8);
      const int64_t row = row0 + r, k = k0 + c;
      bf16 t[8];
      if (k < ke && row + 8 <= row_lim) {
        *reinterpret_cast<uint4*>(t) = __ldg(reinterpret_cast<const uint4*>(src + k * s_k + row));
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) t[i] = (k < ke && row + i < row_lim) ? src[k * s_k + row + i] : zero;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) T[canon(r + i, c)] = t[i];
    }
  } else {
    for (int e = tid; e < rows * kTK; e += kTcThreads) {
      int r, c;
      if (s_k == 1) { r = e / kTK; c = e % kTK; }
      else { c = e / rows; r = e % rows; }
      const int64_t row = row0 + r, k = k0 + c;
      T[canon(r, c)] = (row < row_lim && k < ke) ? src[row * s_row + k * s_k] : zero;
    }
  }
}

// C = A B with A (M x K) and B (K x N) in bf16, FP32 accumulation in tensor
// memory (tcgen05), fused epilogue.  One CTA per 128 x 128 tile of C (and per
// K chunk, blockIdx.z): all 128 threads stage A and B into shared memory in
// the canonical layout (any global strides); one thread issues the four
// K = 16 MMAs of a stage and commits them to an mbarrier; after the last
// stage each warp reads its 32 accumulator rows from tensor memory.
template <int EPI>
__global__ void __launch_bounds__(kTcThreads) k_gemm(const GemmArgs g) {
  __shared__ __align__(128) bf16 As[kTM * kTK];
  __shared__ __align__(128) bf16 Bs[kTN * kTK];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * kTM, n0 = (int64_t)blockIdx.y * kTN;
  const int64_t kb = (int64_t)blockIdx.z * g.kchunk;
  const int64_t ke = g.K < kb + g.kchunk ? g.K : kb + g.kchunk;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) mbar_init1(&bar);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  bool ok = true;
  uint32_t phase = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += kTK) {
    stage_tile(As, g.A, g.sam, g.sak, m0, g.M, k0, ke, kTM, tid);
    stage_tile(Bs, g.B, g.sbn, g.sbk, n0, g.N, k0, ke, kTN, tid);
    // make the generic-proxy stores visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kTK / 16; ++kk) {
        // K = 16 is two core matrices along K: advance the start by 2 LBO
        const uint64_t ad = smem_desc(saddr(As) + kk * 2 * kLBO);
        const uint64_t bd = smem_desc(saddr(Bs) + kk * 2 * kLBO);
        const uint32_t acc = (k0 > kb || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
            : "memory");
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              saddr(&bar))
          : "memory");
    }
    // every thread takes the same branch (the tensor-memory loads below are
    // warp-collective)
    if (!__syncthreads_and(mbar_wait(&bar, phase) ? 1 : 0)) {
      if (tid == 0) atomicOr(g.err, 1);
      mbar_wait(&bar, phase);  // a second bounded chance for the MMAs in flight
      ok = false;
      break;
    }
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok && kb < ke) {
    const int64_t m = m0 + warp * 32 + lane;  // accumulator row = tensor-memory lane
#pragma unroll 1
    for (int c0 = 0; c0 < kTN; c0 += 16) {
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m >= g.M) continue;
      const int64_t nb = n0 + c0;
      float x[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = __uint_as_float(v[j]);
      // Each thread owns 16 consecutive outputs of one row: whole 16-byte
      // vectors when the row segment is full and aligned, else element-wise.
      if constexpr (EPI == kEpiTanh || EPI == kEpiDTanh) {
        bf16* o = g.o16 + m * g.ldo + nb;
        if (nb + 16 <= g.N && ((uintptr_t)o & 15u) == 0 &&
            (EPI == kEpiTanh || ((uintptr_t)(g.hprev + m * g.ldh + nb) & 15u) == 0)) {
          __align__(16) bf16 t[16];
          if constexpr (EPI == kEpiDTanh) {
            __align__(16) bf16 h[16];
            *reinterpret_cast<uint4*>(h) = *reinterpret_cast<const uint4*>(g.hprev + m * g.ldh + nb);
            *reinterpret_cast<uint4*>(h + 8) =
                *reinterpret_cast<const uint4*>(g.hprev + m * g.ldh + nb + 8);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float hv = __bfloat162float(h[j]);
              t[j] = __float2bfloat16_rn(x[j] * (1.0f - hv * hv));
            }
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) t[j] = __float2bfloat16_rn(tanhf(x[j] + g.bias[nb + j]));
          }
          reinterpret_cast<uint4*>(o)[0] = reinterpret_cast<const uint4*>(t)[0];
          reinterpret_cast<uint4*>(o)[1] = reinterpret_cast<const uint4*>(t)[1];
          continue;
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t n = nb + j;
        if (n >= g.N) break;
        if constexpr (EPI == kEpiTanh) {
          g.o16[m * g.ldo + n] = __float2bfloat16_rn(tanhf(x[j] + g.bias[n]));
        } else if constexpr (EPI == kEpiLinear) {
          g.o32[m * g.ldo + n] = x[j] + g.bias[n];
        } else if constexpr (EPI == kEpiDTanh) {
          const float h = __bfloat162float(g.hprev[m * g.ldh + n]);
          g.o16[m * g.ldo + n] = __float2bfloat16_rn(x[j] * (1.0f - h * h));
        } else {
          atomicAdd(g.o32 + m * g.ldo + n, x[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
}

template <int EPI>
int gemm(const GemmArgs& g, int64_t splits, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return 0;
  dim3 grid((unsigned)((g.M + kTM - 1) / kTM), (unsigned)((g.N + kTN - 1) / kTN),
            (unsigned)splits);
  // 15 KB of (unused) dynamic shared memory on top of the 32 KB of tiles caps
  // an SM at 4 CTAs, so their 4 x 128 accumulator columns always fit in the
  // 512 columns of tensor memory and no allocation ever waits.
  k_gemm<EPI><<<grid, kTcThreads, kTcSmemPad, s>>>(g);
  return (int)cudaGetLastError();
}

// ----------------------------------------------------- elementwise kernels

__global__ void k_to_bf16(const float* x, bf16* y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// Output error d = bf16(scale (y - t)) with scale = 2 / count, and the loss
// sum (y - t)^2 / count accumulated into *loss.
__global__ void k_mse(const float* y, const float* t, int64_t count, float scale, bf16* d,
                      double* loss, double inv_count) {
  float s = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float e = y[i] - t[i];
    d[i] = __float2bfloat16_rn(scale * e);
    s += e * e;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)s * inv_count);
}

// out[c] += sum over rows [r0, r1) of d[r][c]: one thread per column.
__global__ void k_colsum(const bf16* d, int64_t rows, int cols, int64_t ld, int64_t per_block,
                         float* out) {
  const int c = threadIdx.x;
  if (c >= cols) return;
  const int64_t r0 = (int64_t)blockIdx.x * per_block;
  const int64_t r1 = rows < r0 + per_block ? rows : r0 + per_block;
  float s = 0.0f;
  for (int64_t r = r0; r < r1; ++r) s += __bfloat162float(d[r * ld + c]);
  atomicAdd(out + c, s);
}

// Adam on the FP32 master parameters; c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void k_adam(float* th, const float* g, float* m, float* v, bf16* w16, int64_t n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = th[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    th[i] = t;
    w16[i] = __float2bfloat16_rn(t);
  }
}

int grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// ------------------------------------------------------- warm-start kernels

struct SiteFrame {
  double s, r;     // axial coordinate from the inlet plane, distance from the axis
  double er[3];    // outward radial unit vector (0 on the axis)
};

__device__ __forceinline__ SiteFrame site_frame(const int32_t* coords, int64_t i,
                                                const lbm_warm_frame& f) {
  const double p[3] = {coords[3 * i] - f.centre[0], coords[3 * i + 1] - f.centre[1],
                       coords[3 * i + 2] - f.centre[2]};
  const double a = p[0] * f.axis[0] + p[1] * f.axis[1] + p[2] * f.axis[2];
  double q[3] = {p[0] - a * f.axis[0], p[1] - a * f.axis[1], p[2] - a * f.axis[2]};
  const double r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  SiteFrame sf;
  sf.s = a - f.z0;
  sf.r = r;
  const double ir = r > 1e-12 ? 1.0 / r : 0.0;
  for (int k = 0; k < 3; ++k) sf.er[k] = q[k] * ir;
  return sf;
}

__global__ void k_warm_features(const int32_t* coords, int64_t n, const lbm_warm_frame f,
                                const double* rho, const double* u, float* x, float* t) {
  const int nin = f.n_global + 2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const SiteFrame sf = site_frame(coords, i, f);
    float* xi = x + i * nin;
    for (int k = 0; k < f.n_global; ++k) xi[k] = f.global[k];
    xi[f.n_global] = (float)(sf.s / f.length);
    xi[f.n_global + 1] = (float)(sf.r / f.radius);
    if (t) {
      const double* ui = u + 3 * i;
      const double ur = ui[0] * sf.er[0] + ui[1] * sf.er[1] + ui[2] * sf.er[2];
      const double uz = ui[0] * f.axis[0] + ui[1] * f.axis[1] + ui[2] * f.axis[2];
      t[3 * i] = (float)((rho[i] - 1.0) / f.rho_scale);
      t[3 * i + 1] = (float)(ur / f.u_scale);
      t[3 * i + 2] = (float)(uz / f.u_scale);
    }
  }
}

__global__ void k_warm_fields(const int32_t* coords, int64_t n, const lbm_warm_frame f,
                              const float* y, double* rho, double* u) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const SiteFrame sf = site_frame(coords, i, f);
    const double ur = f.u_scale * (double)y[3 * i + 1];
    const double uz = f.u_scale * (double)y[3 * i + 2];
    rho[i] = 1.0 + f.rho_scale * (double)y[3 * i];
    for (int k = 0; k < 3; ++k) u[3 * i + k] = ur * sf.er[k] + uz * f.axis[k];
  }
}

}  // namespace

// ------------------------------------------------------------------ network

struct lbm_mlp {
  int n_in = 0, width = 0, n_layers = 0, n_out = 0;
  int64_t max_batch = 0;
  std::vector<int> rows, cols;       // W_l shape
  std::vector<int64_t> w_off, b_off;  // offsets in the parameter vector
  int64_t n_params = 0;
  cudaStream_t stream = nullptr;
  lbm_allocator alloc{};
  bool user_alloc = false;
  std::vector<void*> owned;
  float* theta = nullptr;  // FP32 master parameters
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  bf16* w16 = nullptr;     // bfloat16 copy (same offsets)
  bf16* x16 = nullptr;     // [max_batch][n_in]
  std::vector<bf16*> h;    // h_1 .. h_{L-1}: [max_batch][width]
  float* y = nullptr;      // [max_batch][n_out]
  bf16* d[2] = {nullptr, nullptr};  // errors, [max_batch][max(width, n_out)]
  double* loss = nullptr;
  int* dflag = nullptr;    // device flag: a bounded tensor-core wait gave up
  int64_t t = 0;           // Adam steps taken
  std::string err;
};

namespace {

int mfail(lbm_mlp* net, int code, const std::string& msg) {
  if (net) net->err = msg;
  return code;
}
int mcuda(lbm_mlp* net, int e, const char* what) {
  if (e == 0) return LBM_OK;
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString((cudaError_t)e));
  return mfail(net, LBM_ECUDA, buf);
}

void* malloc_dev(lbm_mlp* net, size_t bytes) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (net->user_alloc) {
    p = net->alloc.alloc(bytes, net->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) net->owned.push_back(p);
  return p;
}

// Layer l reads h_l: the bfloat16 inputs (l = 0) or the activations h[l-1].
const bf16* layer_in(const lbm_mlp* net, int l) { return l == 0 ? net->x16 : net->h[l - 1]; }

// Forward pass of n <= max_batch rows: y [n][n_out] FP32 (y may be any buffer).
int forward_rows(lbm_mlp* net, const float* x, int64_t n, float* y, cudaStream_t s) {
  int e = 0;
  k_to_bf16<<<grid_for(n * net->n_in, 256), 256, 0, s>>>(x, net->x16, n * net->n_in);
  if ((e = (int)cudaGetLastError())) return e;
  for (int l = 0; l < net->n_layers; ++l) {
    GemmArgs g{};
    g.err = net->dflag;
    g.A = layer_in(net, l);
    g.sam = net->cols[l];
    g.sak = 1;
    g.B = net->w16 + net->w_off[l];
    g.sbk = 1;
    g.sbn = net->cols[l];
    g.M = n;
    g.N = net->rows[l];
    g.K = net->cols[l];
    g.kchunk = g.K;
    g.bias = net->theta + net->b_off[l];
    if (l < net->n_layers - 1) {
      g.o16 = net->h[l];
      g.ldo = net->width;
      e = gemm<kEpiTanh>(g, 1, s);
    } else {
      g.o32 = y;
      g.ldo = net->n_out;
      e = gemm<kEpiLinear>(g, 1, s);
    }
    if (e) return e;
  }
  return 0;
}

// Loss and gradient of the batch into net->loss and net->grad (forward included).
int loss_grad_rows(lbm_mlp* net, const float* x, const float* t, int64_t n, cudaStream_t s) {
  int e = forward_rows(net, x, n, net->y, s);
  if (e) return e;
  if ((e = (int)cudaMemsetAsync(net->grad, 0, net->n_params * sizeof(float), s))) return e;
  if ((e = (int)cudaMemsetAsync(net->loss, 0, sizeof(double), s))) return e;
  const int64_t count = n * net->n_out;
  k_mse<<<grid_for(count, 256), 256, 0, s>>>(net->y, t, count, (float)(2.0 / (double)count),
                                              net->d[0], net->loss, 1.0 / (double)count);
  if ((e = (int)cudaGetLastError())) return e;
  int cur = 0;
  // Row splits of the weight-gradient contraction (over the batch).
  const int64_t chunk = 2048;
  const int64_t splits = (n + chunk - 1) / chunk;
  for (int l = net->n_layers - 1; l >= 0; --l) {
    const int64_t ldd = net->rows[l];  // columns of the current error d_l
    const bf16* dl = net->d[cur];
    // dW_l = d_l^T h_l: [rows][cols], contraction over the n rows.
    GemmArgs gw{};
    gw.err = net->dflag;
    gw.A = dl;
    gw.sam = 1;
    gw.sak = ldd;
    gw.B = layer_in(net, l);
    gw.sbk = net->cols[l];
    gw.sbn = 1;
    gw.M = net->rows[l];
    gw.N = net->cols[l];
    gw.K = n;
    gw.kchunk = chunk;
    gw.o32 = net->grad + net->w_off[l];
    gw.ldo = net->cols[l];
    if ((e = gemm<kEpiAccum>(gw, splits, s))) return e;
    // db_l = column sums of d_l.
    const int64_t per = 512;
    const int threads = ((net->rows[l] + 31) / 32) * 32;
    k_colsum<<<(unsigned)((n + per - 1) / per), threads, 0, s>>>(dl, n, net->rows[l], ldd, per,
                                                                 net->grad + net->b_off[l]);
    if ((e = (int)cudaGetLastError())) return e;
    if (l == 0) break;
    // d_{l-1} = (d_l W_l) * (1 - h_l^2): [n][cols_l].
    GemmArgs gd{};
    gd.err = net->dflag;
    gd.A = dl;
    gd.sam = ldd;
    gd.sak = 1;
    gd.B = net->w16 + net->w_off[l];
    gd.sbk = net->cols[l];
    gd.sbn = 1;
    gd.M = n;
    gd.N = net->cols[l];
    gd.K = net->rows[l];
    gd.kchunk = gd.K;
    gd.hprev = layer_in(net, l);
    gd.ldh = net->cols[l];
    gd.o16 = net->d[cur ^ 1];
    gd.ldo = net->cols[l];
    if ((e = gemm<kEpiDTanh>(gd, 1, s))) return e;
    cur ^= 1;
  }
  return 0;
}

int copy_kind(int32_t device_side, bool to_device) {
  if (device_side) return cudaMemcpyDeviceToDevice;
  return to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
}

}  // namespace

namespace lbm {

int mlp_forward_on(lbm_mlp* net, const float* x, int64_t n, float* y, void* stream) {
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t r = 0; r < n; r += net->max_batch) {
    const int64_t m = std::min(net->max_batch, n - r);
    const int e = forward_rows(net, x + r * net->n_in, m, y + r * net->n_out, s);
    if (e) return e;
  }
  return 0;
}

void mlp_shape(const lbm_mlp* net, int* n_in, int* n_out, void** stream) {
  *n_in = net->n_in;
  *n_out = net->n_out;
  *stream = net->stream;
}

int launch_warm_features(const int32_t* coords, int64_t n, const lbm_warm_frame& f,
                         const double* rho, const double* u, float* x, float* t, void* stream) {
  if (n <= 0) return 0;
  k_warm_features<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(coords, n, f,
                                                                                    rho, u, x, t);
  return (int)cudaGetLastError();
}

int launch_warm_fields(const int32_t* coords, int64_t n, const lbm_warm_frame& f, const float* y,
                       double* rho, double* u, void* stream) {
  if (n <= 0) return 0;
  k_warm_fields<<<grid_for(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(coords, n, f, y,
                                                                                  rho, u);
  return (int)cudaGetLastError();
}

}  // namespace lbm

extern "C" {

int lbm_mlp_create(int32_t n_in, int32_t width, int32_t n_layers, int32_t n_out,
                   int64_t max_batch, const lbm_allocator* alloc, void* cuda_stream,
                   lbm_mlp** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (n_in < 1 || n_in > LBM_MLP_MAX_IN || width < 1 || width > LBM_MLP_MAX_WIDTH ||
      n_layers < 1 || n_layers > 64 || n_out < 1 || n_out > LBM_MLP_MAX_OUT || max_batch < 1 ||
      max_batch > ((int64_t)1 << 31) / LBM_MLP_MAX_WIDTH)
    return LBM_EINVAL;
  if (alloc && (!alloc->alloc || !alloc->free)) return LBM_EINVAL;
  lbm_mlp* net = new (std::nothrow) lbm_mlp;
  if (!net) return LBM_ENOMEM;
  net->n_in = n_in;
  net->width = width;
  net->n_layers = n_layers;
  net->n_out = n_out;
  net->max_batch = max_batch;
  net->stream = static_cast<cudaStream_t>(cuda_stream);
  if (alloc) {
    net->alloc = *alloc;
    net->user_alloc = true;
  }
  int64_t o = 0;
  for (int l = 0; l < n_layers; ++l) {
    const int r = l == n_layers - 1 ? n_out : width;
    const int c = l == 0 ? n_in : width;
    net->rows.push_back(r);
    net->cols.push_back(c);
    net->w_off.push_back(o);
    o += (int64_t)r * c;
    net->b_off.push_back(o);
    o += r;
  }
  net->n_params = o;
  bool ok = true;
  auto f32 = [&](int64_t count) {
    float* p = static_cast<float*>(malloc_dev(net, count * sizeof(float)));
    ok = ok && p;
    return p;
  };
  auto b16 = [&](int64_t count) {
    bf16* p = static_cast<bf16*>(malloc_dev(net, count * sizeof(bf16)));
    ok = ok && p;
    return p;
  };
  net->theta = f32(o);
  net->grad = f32(o);
  net->m = f32(o);
  net->v = f32(o);
  net->w16 = b16(o);
  net->x16 = b16(max_batch * n_in);
  for (int l = 0; l + 1 < n_layers; ++l) net->h.push_back(b16(max_batch * width));
  net->y = f32(max_batch * n_out);
  const int dw = std::max(width, n_out);
  net->d[0] = b16(max_batch * dw);
  net->d[1] = b16(max_batch * dw);
  net->loss = static_cast<double*>(malloc_dev(net, sizeof(double)));
  net->dflag = static_cast<int*>(malloc_dev(net, sizeof(int)));
  ok = ok && net->loss && net->dflag;
  if (!ok) {
    lbm_mlp_destroy(net);
    return LBM_ENOMEM;
  }
  cudaStream_t s = net->stream;
  int e = 0;
  for (void* p : {(void*)net->theta, (void*)net->grad, (void*)net->m, (void*)net->v})
    if (!e) e = (int)cudaMemsetAsync(p, 0, o * sizeof(float), s);
  if (!e) e = (int)cudaMemsetAsync(net->w16, 0, o * sizeof(bf16), s);
  if (!e) e = (int)cudaMemsetAsync(net->dflag, 0, sizeof(int), s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  if (e) {
    lbm_mlp_destroy(net);
    return LBM_ECUDA;
  }
  *out = net;
  return LBM_OK;
}

int lbm_mlp_param_count(const lbm_mlp* net, int64_t* count) {
  if (!net || !count) return LBM_EINVAL;
  *count = net->n_params;
  return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp* net, const float* theta, int32_t src_is_device) {
  if (!net) return LBM_EINVAL;
  if (!theta) return mfail(net, LBM_EINVAL, "lbm_mlp_set_params: NULL parameters");
  cudaStream_t s = net->stream;
  const size_t bytes = net->n_params * sizeof(float);
  int e = (int)cudaMemcpyAsync(net->theta, theta, bytes,
                               (cudaMemcpyKind)copy_kind(src_is_device, true), s);
  if (!e) e = (int)cudaMemsetAsync(net->m, 0, bytes, s);
  if (!e) e = (int)cudaMemsetAsync(net->v, 0, bytes, s);
  if (!e) {
    k_to_bf16<<<grid_for(net->n_params, 256), 256, 0, s>>>(net->theta, net->w16, net->n_params);
    e = (int)cudaGetLastError();
  }
  if (!e) e = (int)cudaStreamSynchronize(s);
  net->t = 0;
  return mcuda(net, e, "lbm_mlp_set_params");
}

int lbm_mlp_get_params(lbm_mlp* net, float* theta, int32_t dst_is_device) {
  if (!net) return LBM_EINVAL;
  if (!theta) return mfail(net, LBM_EINVAL, "lbm_mlp_get_params: NULL output");
  int e = (int)cudaMemcpyAsync(theta, net->theta, net->n_params * sizeof(float),
                               (cudaMemcpyKind)copy_kind(dst_is_device, false), net->stream);
  if (!e && !dst_is_device) e = (int)cudaStreamSynchronize(net->stream);
  return mcuda(net, e, "lbm_mlp_get_params");
}

int lbm_mlp_forward(lbm_mlp* net, const float* x, int64_t n, float* y) {
  if (!net) return LBM_EINVAL;
  if (n < 0 || (n > 0 && (!x || !y))) return mfail(net, LBM_EINVAL, "lbm_mlp_forward: arguments");
  return mcuda(net, lbm::mlp_forward_on(net, x, n, y, net->stream), "lbm_mlp_forward");
}

int lbm_mlp_loss_grad(lbm_mlp* net, const float* x, const float* t, int64_t n, double* loss,
                      float* grad, int32_t dst_is_device) {
  if (!net) return LBM_EINVAL;
  if (!x || !t || !loss || n < 1 || n > net->max_batch)
    return mfail(net, LBM_EINVAL, "lbm_mlp_loss_grad: arguments");
  cudaStream_t s = net->stream;
  int e = loss_grad_rows(net, x, t, n, s);
  if (!e && grad)
    e = (int)cudaMemcpyAsync(grad, net->grad, net->n_params * sizeof(float),
                             (cudaMemcpyKind)copy_kind(dst_is_device, false), s);
  if (!e) e = (int)cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (!e) e = (int)cudaStreamSynchronize(s);
  return mcuda(net, e, "lbm_mlp_loss_grad");
}

int lbm_mlp_train_step(lbm_mlp* net, const float* x, const float* t, int64_t n,
                       const lbm_adam* opt, double* loss) {
  if (!net) return LBM_EINVAL;
  if (!x || !t || !opt || n < 1 || n > net->max_batch || !(opt->lr >= 0.0) ||
      !(opt->beta1 >= 0.0 && opt->beta1 < 1.0) || !(opt->beta2 >= 0.0 && opt->beta2 < 1.0) ||
      !(opt->eps > 0.0))
    return mfail(net, LBM_EINVAL, "lbm_mlp_train_step: arguments");
  cudaStream_t s = net->stream;
  int e = loss_grad_rows(net, x, t, n, s);
  if (e) return mcuda(net, e, "lbm_mlp_train_step");
  net->t += 1;
  const double c1 = 1.0 / (1.0 - std::pow(opt->beta1, (double)net->t));
  const double c2 = 1.0 / (1.0 - std::pow(opt->beta2, (double)net->t));
  k_adam<<<grid_for(net->n_params, 256), 256, 0, s>>>(
      net->theta, net->grad, net->m, net->v, net->w16, net->n_params, (float)opt->lr,
      (float)opt->beta1, (float)opt->beta2, (float)opt->eps, (float)c1, (float)c2);
  e = (int)cudaGetLastError();
  if (!e && loss) {
    e = (int)cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (!e) e = (int)cudaStreamSynchronize(s);
  }
  return mcuda(net, e, "lbm_mlp_train_step");
}

int lbm_mlp_sync(lbm_mlp* net) {
  if (!net) return LBM_EINVAL;
  int rc = mcuda(net, (int)cudaStreamSynchronize(net->stream), "lbm_mlp_sync");
  if (rc != LBM_OK) return rc;
  int flag = 0;
  int e = (int)cudaMemcpyAsync(&flag, net->dflag, sizeof(int), cudaMemcpyDeviceToHost, net->stream);
  if (!e) e = (int)cudaStreamSynchronize(net->stream);
  if (e) return mcuda(net, e, "lbm_mlp_sync flag");
  if (flag) {
    cudaMemsetAsync(net->dflag, 0, sizeof(int), net->stream);
    cudaStreamSynchronize(net->stream);
    return mfail(net, LBM_ETIMEOUT, "a bounded wait for the tensor cores gave up");
  }
  return LBM_OK;
}

const char* lbm_mlp_last_error(const lbm_mlp* net) { return net ? net->err.c_str() : ""; }

void lbm_mlp_destroy(lbm_mlp* net) {
  if (!net) return;
  cudaStreamSynchronize(net->stream);
  for (void* p : net->owned) {
    if (net->user_alloc) net->alloc.free(p, net->alloc.user);
    else cudaFree(p);
  }
  delete net;
}

}  // extern "C"
