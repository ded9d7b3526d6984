// tcgen05 / TMA / mbarrier building blocks for sm_103a shared by the
// tensor-core kernels (the surrogate's forward and backward passes): the
// instruction and shared-memory descriptors of kind::f16 MMAs on K-major
// bf16 operands in the 128-byte swizzled layout that TMA writes, bounded
// mbarrier waits, TMEM loads and packed fp32x2 arithmetic.  Everything lives
// in an unnamed namespace, so each translation unit gets its own copy.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "wh_internal.h"

namespace wh {
namespace {

// instruction descriptor of tcgen05.mma kind::f16: fp32 accumulator (bits
// 4-5), A and B bf16 (bits 7-9, 10-12), both K-major (bits 15, 16 clear),
// N/8 at bits 17-22, M/16 at bits 24-28
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);

constexpr unsigned long long WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete.  Gives up when the CTA's abort
// flag is set or after wait_ns (default WAIT_NS), setting the flag and the
// status word.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, int* status,
                                       unsigned long long wait_ns = WAIT_NS) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*abort) return false;
            if (globaltimer() - t0 > wait_ns || i > (1u << 30)) {
                *abort = 1;
                atomicOr(status, (int)WH_STATUS_TIMEOUT);
                return false;
            }
        }
    }
}

// used after an abort: wait for a phase without giving up on the flag
__device__ void mbar_drain(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 0; !mbar_try(bar, parity); ++i)
        if ((i & 63) == 0 && globaltimer() - t0 > WAIT_NS) return;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that TMA writes: 8-row groups 1024 bytes apart (stride
// byte offset), descriptor version 1 (bit 46), swizzle mode 2 (bits 61-63).
// Advancing K by 16 bf16 inside a 1024-byte aligned atom adds 32 bytes to
// the start address.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// 32 TMEM lanes x 32 fp32 columns: lane i of the warp receives its lane's
// columns [col, col + 32).  The wait names the registers so that no use of
// them is scheduled before the load has landed.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 TMEM lanes x 16 fp32 columns (lane i of the warp receives its lane's
// columns [col, col + 16)); as tc_ld32.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Split forms of tc_ld16 for software pipelining: tc_ld16_issue starts the
// load of 16 columns into r; tc_wait_ld16 waits for every load of the warp
// issued so far and names r, so that no use of r is scheduled before it.
__device__ __forceinline__ void tc_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tc_wait_ld16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// Pairs of fp32 values in one 64-bit register for the packed fp32x2
// arithmetic of sm_100 and later (add / mul / fma .f32x2, element-wise,
// round to nearest): the epilogue's FMA-pipe work in half the instructions.
__device__ __forceinline__ uint64_t pk(float lo, float hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(uint64_t r, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t dup2(float x) { return pk(x, x); }

// gelu(z) = z/2 (1 + erf(z / sqrt 2)) of both halves of z, with erf by the
// approximation of Abramowitz & Stegun, Handbook of Mathematical Functions,
// formula 7.1.28 (after Hastings): for x >= 0,
// erf(x) = 1 - P(x)^-16, P(x) = 1 + a1 x + ... + a6 x^6, |error| <= 3e-7;
// odd in x.  Both signs of z reduce to one expression,
//   gelu(z) = relu(z) - |z| P(|z| / sqrt 2)^-16 / 2 = relu(z) - |z| Q(|z|)^-16,
// with Q(t) = c P(t / sqrt 2), c = 2^(1/16) (so Q^16 = 2 P^16): coefficients
// q_k = c a_k / sqrt(2)^k, all positive.  Error of the fp32 evaluation: the
// Horner chain over positive terms and the rounded coefficients perturb Q by
// at most 7u relative (u = 2^-24), the four squarings make that 127u, the
// reciprocal 129u, the product with |z| 130u of a term of at most |z|/2, and
// the final fma adds u |z|: at most 66u |z|, plus the approximation's own
// 1.5e-7 |z|.  Large |z|: Q^16 overflows, the reciprocal is 0 and
// gelu = relu(z).  All but the two reciprocals on packed pairs.
constexpr float GELU_Q0 = 1.0442737f, GELU_Q1 = 0.052075163f, GELU_Q2 = 0.022076998f,
                GELU_Q3 = 0.0034227392f, GELU_Q4 = 3.9686136e-05f, GELU_Q5 = 5.105521e-05f,
                GELU_Q6 = 5.6213e-06f;

__device__ __forceinline__ uint64_t gelu2(uint64_t z) {
    float z0, z1;
    upk(z, z0, z1);
    const uint64_t t = pk(fabsf(z0), fabsf(z1));
    uint64_t q = fma2(dup2(GELU_Q6), t, dup2(GELU_Q5));
    q = fma2(q, t, dup2(GELU_Q4));
    q = fma2(q, t, dup2(GELU_Q3));
    q = fma2(q, t, dup2(GELU_Q2));
    q = fma2(q, t, dup2(GELU_Q1));
    q = fma2(q, t, dup2(GELU_Q0));
    q = mul2(q, q);   // ^2
    q = mul2(q, q);   // ^4
    q = mul2(q, q);   // ^8
    q = mul2(q, q);   // ^16
    float p0, p1;
    upk(q, p0, p1);
    const uint64_t nr = pk(-1.0f / p0, -1.0f / p1);
    return fma2(t, nr, pk(fmaxf(z0, 0.0f), fmaxf(z1, 0.0f)));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&p);
}

}  // namespace
}  // namespace wh
