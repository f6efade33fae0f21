// tcgen05 pieces shared by the kernels that issue 5th-generation tensor-core
// MMAs (umma_forward.cu: vertical pass on tcgen05; tc05_forward.cu: both
// passes): shared-memory matrix descriptors, the f16 MMA with its commit,
// tensor-memory loads and the Hankel tap strips the B operands read.
#pragma once

#include "tc_common.cuh"

namespace fovea {
namespace tcc {

constexpr int kXOff = 8;  // strip entry j holds Hankel index X = j - kXOff
__host__ __device__ inline int strip_entries(int rmax) { return rmax / 4 + 16; }

// ---------------------------------------------------------------- tcgen05

// Shared-memory matrix descriptor, no swizzle: core matrices of 8 rows x 16
// bytes (128 contiguous bytes). lbo / sbo are the byte distances between
// core matrices adjacent in K / in M (or N), for a K-major operand (rows
// along M or N, 8 K values per row) and for an MN-major one (rows along K,
// 8 M or N values per row; the transpose bit of the instruction descriptor
// set) alike. Bits 46-48 hold the descriptor version 1.
__device__ __forceinline__ unsigned long long umma_desc(const void* p, unsigned int lbo, unsigned int sbo) {
  const unsigned int a = smem_u32(p);
  return (unsigned long long)((a & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void umma_f16(unsigned int d_tmem, unsigned long long a, unsigned long long b,
                                         unsigned int idesc, unsigned int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrives on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void umma_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc05_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc05_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(unsigned int taddr, float (&d)[32]) {
  unsigned int u[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]),
        "=r"(u[24]), "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
  #pragma unroll
  for (int i = 0; i < 32; ++i) d[i] = __uint_as_float(u[i]);
}

// Hankel strip of one item for pass 1: entry j is two 128-byte core
// matrices, hi then lo, whose row rho, column i holds the hi / lo fp16 part
// of the scaled tap u(8 (j - kXOff) + rho + i + delta) * 2^12. Read with N
// groups 128 bytes apart and K groups 256 bytes apart, N group 2a' + p of
// the MMA's B is part p (hi, lo) of the Hankel core matrix a' + b: one
// N = 64 instruction computes both products.
template <int NT = kThreads>
__device__ __forceinline__ void make_strips(__half* S2, int nent, int r, float c, float S, int delta,
                                            int t0 = threadIdx.x) {
  for (int idx = t0; idx < nent * 32; idx += NT) {
    const int j = idx >> 5, rho = (idx >> 2) & 7, i0 = (idx & 3) * 2;
    const int m0 = 8 * (j - kXOff) + rho + i0 + delta;
    const float w0 = tap_u(m0, r, c, S) * kWScale, w1 = tap_u(m0 + 1, r, c, S) * kWScale;
    const __half h0 = __float2half_rn(w0), h1 = __float2half_rn(w1);
    const __half l0 = __float2half_rn(w0 - __half2float(h0)), l1 = __float2half_rn(w1 - __half2float(h1));
    const int o = j * 128 + rho * 8 + i0;
    *reinterpret_cast<unsigned int*>(S2 + o) = pack_half2(h0, h1);
    *reinterpret_cast<unsigned int*>(S2 + o + 64) = pack_half2(l0, l1);
  }
}


// Normalised taps of one item, u(m) for m in [0, 2r], into U (NT threads):
// the same values tap_u gives, computed once so that the tap strips and the
// cumulative sums read them instead of evaluating exp again.
template <int NT>
__device__ __forceinline__ void make_tap_table(float* U, int r, float c, float S) {
  for (int m = threadIdx.x; m <= 2 * r; m += NT) U[m] = tap_u(m, r, c, S);
}

__device__ __forceinline__ float tap_at(const float* U, int m, int r) { return (m >= 0 && m <= 2 * r) ? U[m] : 0.0f; }

// make_strips from a tap table: one thread per (entry, row), the row's 8
// taps as one 16-byte store each of the hi and the lo parts.
template <int NT>
__device__ __forceinline__ void make_strips_tab(__half* S2, int nent, const float* U, int r, int delta) {
  for (int idx = threadIdx.x; idx < nent * 8; idx += NT) {
    const int j = idx >> 3, rho = idx & 7;
    const int m0 = 8 * (j - kXOff) + rho + delta;
    unsigned int hw[4], lw[4];
    #pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float w0 = tap_at(U, m0 + 2 * i, r) * kWScale, w1 = tap_at(U, m0 + 2 * i + 1, r) * kWScale;
      const __half h0 = __float2half_rn(w0), h1 = __float2half_rn(w1);
      hw[i] = pack_half2(h0, h1);
      lw[i] = pack_half2(__float2half_rn(w0 - __half2float(h0)), __float2half_rn(w1 - __half2float(h1)));
    }
    __half* o = S2 + j * 128 + rho * 8;
    *reinterpret_cast<uint4*>(o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(o + 64) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// make_cumulative_tc from a tap table (one warp; the same summation order).
__device__ __forceinline__ void make_cumulative_tab(float* CU, const float* U, int r) {
  const int lane = threadIdx.x & 31;
  const int n = 2 * r + 1;
  const int seg = (n + 31) >> 5;
  const int b = lane * seg, e = min(n, b + seg);
  float sum = 0.0f;
  for (int m = b; m < e; ++m) sum += U[m];
  float incl = sum;
  #pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  float run = incl - sum;
  for (int m = b; m < e; ++m) {
    CU[m] = run;
    run += U[m];
  }
  if (lane == 31) CU[n] = incl;
}

}  // namespace tcc
}  // namespace fovea
