// storm_mlp.cuh -- the self-collision surrogate network on Blackwell tensor cores.
//
// The paper replaces its exact self-collision check by a learned distance
// network (Sec. 4.2, Eq. 13).  Here: 16 encoded inputs -> 256 -> 256 -> 256 -> 1
// with ReLU, BF16 operands and FP32 accumulation.  Every GEMM runs on the 5th
// generation tensor cores: operands staged in shared memory (by cp.async in the
// no-swizzle K-major core-matrix layout, or, for the warp-specialised layer
// kernel's 64-column K tiles, by TMA tensor loads in the 128-byte swizzled
// layout), one elected thread issues tcgen05.mma with the accumulator in tensor
// memory (TMEM), tcgen05.commit signals an mbarrier, and the epilogue reads TMEM
// with tcgen05.ld (the layer kernel writes its tiles back by TMA tensor
// stores).  Every wait is bounded in time and reports through an error flag.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

namespace tc {

constexpr int kBM = 128;         // rows of a CTA tile = TMEM lanes
constexpr int kKB = 64;          // K per shared-memory stage
constexpr int kThreads = 128;    // one warpgroup: warp w owns TMEM lanes 32w..32w+31
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s bound on any wait

struct GemmArgs {
    const __nv_bfloat16* A;  // M x K, row-major (K contiguous)
    const __nv_bfloat16* B;  // N x K, row-major (K contiguous)
    int lda, ldb;
    int M, N, K;             // M % 128 == 0, N % 16 == 0 and <= 256, K % 16 == 0
    const float* bias;       // N (nullable)
    int relu;
    const __nv_bfloat16* mask;  // M x N: keep entries where mask > 0 (nullable)
    int ldm;
    __nv_bfloat16* out_bf;      // M x N (nullable)
    int ldo;
    __nv_bfloat16* out_bfT;     // N x M (nullable)
    int ldoT;
    float* out_f;               // M x N (nullable)
    int ldf;
    const float* head_w;        // N: y[m] = *head_b + sum_n head_w[n] v[m][n] (nullable)
    const float* head_b;
    float* head_y;              // M
    int* err;                   // set to 1 when a wait times out
    size_t split_stride;        // split-K: CTA row blockIdx.y takes K range [y K, (y+1) K) of A and B
                                // and writes out_f + y split_stride (0: no split)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor, no swizzle: start address, leading-dimension
// byte offset (between core matrices along K), stride-dimension byte offset
// (between 8-row groups), the fixed 0b001 at bits 46-48.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) |
           (static_cast<uint64_t>((lbo & 0x3FFFFu) >> 4) << 16) |
           (static_cast<uint64_t>((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

// Descriptor of a K-major operand in the 128-byte swizzled layout that TMA
// writes: rows of 64 BF16 (128 bytes), 16-byte chunk c of row r at chunk
// c ^ (r mod 8), 8-row groups 1024 bytes apart (the stride field; the leading
// field is unused for this layout), layout code 2 at bits 61-63; the K steps of
// 16 elements advance the start address by 32 bytes within the rows.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr)
{
    return static_cast<uint64_t>((addr & 0x3FFFFu) >> 4) | (1ull << 16) | (static_cast<uint64_t>(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// Bulk tensor load (TMA) of the box at element coordinates (x, y) of the tensor
// map's 2-D view into shared memory, completing its bytes on mbarrier mbar.
__device__ __forceinline__ void tma_load_2d(const CUtensorMap* map, uint32_t dst, uint32_t mbar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(y)
        : "memory");
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, N, M.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

// One non-blocking probe: has the phase with parity `parity` completed?
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with parity `parity` to complete; false once limit_ns
// nanoseconds of %globaltimer have passed without it.  A phase that has
// already completed costs one probe; the timer (slow to read) is read only
// once the wait is real, and then every 64 probes.
__device__ __forceinline__ bool mbar_wait_for(uint32_t addr, uint32_t parity, unsigned long long limit_ns)
{
    if (mbar_try(addr, parity)) return true;
    const unsigned long long t0 = now_ns();
    for (uint32_t n = 1;; ++n) {
        if (mbar_try(addr, parity)) return true;
        if ((n & 63u) == 0u && now_ns() - t0 > limit_ns) return false;
    }
}

// The bound every tensor-core wait of the library uses.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    return mbar_wait_for(addr, parity, kWaitNs);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Stage a rows x kb tile (row-major source, K contiguous) into the core-matrix
// layout: element (r, k) at (r / 8) * SBO + (r % 8) * 16 + (k / 8) * 128 + (k % 8) * 2.
__device__ __forceinline__ void stage_tile(uint32_t dst, const __nv_bfloat16* src, int ld, int rows,
                                           int kb)
{
    const int chunks = kb / 8, sbo = chunks * 128;
    for (int c = threadIdx.x; c < rows * chunks; c += blockDim.x) {
        const int r = c / chunks, kg = c - r * chunks;
        cp_async16(dst + (r >> 3) * sbo + (r & 7) * 16 + kg * 128, src + static_cast<size_t>(r) * ld + kg * 8);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// C = A B^T on one 128 x BN tile per CTA, FP32 accumulator in TMEM, fused
// epilogue (bias, ReLU, mask, BF16 / FP32 stores, transposed store, dot head).
template <int BN>
__global__ void __launch_bounds__(kThreads, 1) k_gemm(GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    constexpr int kCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    constexpr int kStageA = kBM * kKB * 2, kStageB = BN * kKB * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM;
    unsigned char* sA[2] = {smem, smem + kStageA + kStageB};
    unsigned char* sB[2] = {smem + kStageA, smem + 2 * kStageA + kStageB};

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const int nk = (g.K + kKB - 1) / kKB;
    uint32_t parity[2] = {0u, 0u};
    bool ok = true;
    const size_t k_base = static_cast<size_t>(blockIdx.y) * g.K;
    const __nv_bfloat16* A = g.A + static_cast<size_t>(m0) * g.lda + k_base;
    const __nv_bfloat16* B = g.B + k_base;
    float* out_f = g.out_f ? g.out_f + blockIdx.y * g.split_stride : nullptr;
    stage_tile(smem_u32(sA[0]), A, g.lda, kBM, min(kKB, g.K));
    stage_tile(smem_u32(sB[0]), B, g.ldb, BN, min(kKB, g.K));
    int last = 0;
    for (int it = 0; it < nk && ok; ++it) {
        const int s = it & 1, k0 = it * kKB, kb = min(kKB, g.K - k0);
        if (it + 1 < nk) {
            const int s2 = s ^ 1, k1 = k0 + kKB, kb1 = min(kKB, g.K - k1);
            if (it >= 1) {  // the MMAs of iteration it-1 read stage s2
                ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[s2]), parity[s2]));
                parity[s2] ^= 1u;
                if (!ok) break;  // uniform across the CTA
            }
            stage_tile(smem_u32(sA[s2]), A + k1, g.lda, kBM, kb1);
            stage_tile(smem_u32(sB[s2]), B + k1, g.ldb, BN, kb1);
            asm volatile("cp.async.wait_group 2;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sbo = (kb / 8) * 128;
            const uint32_t idesc = instr_desc(kBM, BN);
            for (int kk = 0; kk < kb / 16; ++kk) {
                const uint64_t da = smem_desc(smem_u32(sA[s]) + kk * 256, 128, sbo);
                const uint64_t db = smem_desc(smem_u32(sB[s]) + kk * 256, 128, sbo);
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[s]))
                : "memory");
        }
        last = s;
    }
    // every thread waits for the final commit (it covers all earlier MMAs)
    if (ok) ok = mbar_wait(smem_u32(&mbar[last]), parity[last]);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (g.err && lane == 0) atomicExch(g.err, 1);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        mbar_wait(smem_u32(&mbar[last]), parity[last]);  // once more, bounded
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (ok) {
        const int row = m0 + warp * 32 + lane;
        float yacc = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 8) {
            uint32_t r[8];
            const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = c0 + i;
                float x = __uint_as_float(r[i]);
                if (g.bias) x += g.bias[n];
                if (g.relu) x = fmaxf(x, 0.f);
                if (g.mask && !(__bfloat162float(g.mask[static_cast<size_t>(row) * g.ldm + n]) > 0.f)) x = 0.f;
                v[i] = x;
                if (g.head_w) yacc = fmaf(g.head_w[n], x, yacc);
            }
            if (out_f) {
                float4* o = reinterpret_cast<float4*>(out_f + static_cast<size_t>(row) * g.ldf + c0);
                o[0] = make_float4(v[0], v[1], v[2], v[3]);
                o[1] = make_float4(v[4], v[5], v[6], v[7]);
            }
            if (g.out_bf) {
                __align__(16) __nv_bfloat16 b[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) b[i] = __float2bfloat16_rn(v[i]);
                *reinterpret_cast<uint4*>(g.out_bf + static_cast<size_t>(row) * g.ldo + c0) =
                    *reinterpret_cast<const uint4*>(b);
            }
            if (g.out_bfT) {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    g.out_bfT[static_cast<size_t>(c0 + i) * g.ldoT + row] = __float2bfloat16_rn(v[i]);
            }
        }
        if (g.head_w) g.head_y[row] = *g.head_b + yacc;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

template <int BN>
constexpr size_t gemm_smem() { return 2 * (kBM * kKB * 2 + BN * kKB * 2); }

// Layers with N = BN (64, 128 or 256): the whole weight matrix B (BN x K, K <= 256) stays
// resident in shared memory, one persistent CTA per SM walks the 128-row tiles
// of A through a kStagesRW-deep cp.async pipeline, and one elected thread
// issues the tcgen05.mma of each K block.  The accumulator is double-buffered
// in TMEM (2 x 256 columns), so the epilogue of tile t runs while the tensor
// core works on tile t+1; a K block's stage is refilled as soon as the commit
// of its MMAs arrives.  Same epilogue as k_gemm.
constexpr int kStagesRW = 4;

__host__ __device__ constexpr size_t gemm_rw_smem(int BN, int K)
{
    return static_cast<size_t>(BN) * K * 2 + static_cast<size_t>(kStagesRW) * kBM * (K < kKB ? K : kKB) * 2;
}

// TMEM -> registers, 32 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The same load without its wait: the registers are valid after tmem_ld_wait
// on them (which waits for every load this thread has issued), so a thread
// can work on one block while the next is in flight.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])::"memory");
}

// One 32-column block of the epilogue (this thread: row `row`, its 32 TMEM
// values r): bias, ReLU and mask into v, and the dot head's running sums (each
// half of the columns summed in column order, the halves added at the end: the
// order of the whole-network tile's two epilogue warps).
// kShared: bias and head_w are 16-byte aligned shared-memory vectors, read as
// float4 broadcasts (otherwise any pointers, read element by element).
__device__ __forceinline__ float4 lds4(const float* p)
{
    float4 x;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w)
                 : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(p))));
    return x;
}

template <int BN, bool kShared = false>
__device__ __forceinline__ void epilogue_block(const GemmArgs& g, const uint32_t (&r)[32], int row, int c0,
                                               const float* bias, const float* head_w, float (&v)[32],
                                               float& yacc, float& yacc0)
{
    if (kShared) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 b = bias ? lds4(bias + c0 + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float bq[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                float x = __uint_as_float(r[4 * q + l]);
                if (bias) x += bq[l];
                if (g.relu) x = fmaxf(x, 0.f);
                v[4 * q + l] = x;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int n = c0 + i;
            float x = __uint_as_float(r[i]);
            if (bias) x += bias[n];
            if (g.relu) x = fmaxf(x, 0.f);
            v[i] = x;
        }
    }
    if (g.mask) {
        const uint4* mk = reinterpret_cast<const uint4*>(g.mask + static_cast<size_t>(row) * g.ldm + c0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 w = mk[q];
            const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&w);
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (!(__bfloat162float(mb[i]) > 0.f)) v[q * 8 + i] = 0.f;
        }
    }
    if (head_w) {
        if (c0 == BN / 2) {
            yacc0 = yacc;
            yacc = 0.f;
        }
        if (kShared) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 w = lds4(head_w + c0 + 4 * q);
                yacc = fmaf(w.x, v[4 * q], yacc);
                yacc = fmaf(w.y, v[4 * q + 1], yacc);
                yacc = fmaf(w.z, v[4 * q + 2], yacc);
                yacc = fmaf(w.w, v[4 * q + 3], yacc);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) yacc = fmaf(head_w[c0 + i], v[i], yacc);
        }
    }
    if (g.out_f) {
        float4* o = reinterpret_cast<float4*>(g.out_f + static_cast<size_t>(row) * g.ldf + c0);
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

// Epilogue of one 128-row tile (this thread: row `row`, TMEM lanes of `warp`):
// bias, ReLU, mask, BF16 / FP32 / transposed stores and the dot head, 32
// columns per TMEM load.
template <int BN>
__device__ __forceinline__ void gemm_epilogue(const GemmArgs& g, uint32_t tmem, int row, int warp,
                                              const float* bias, const float* head_w)
{
    float yacc = 0.f, yacc0 = 0.f;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, r);
        float v[32];
        epilogue_block<BN>(g, r, row, c0, bias, head_w, v, yacc, yacc0);
        if (g.out_bf) {
            uint4* o = reinterpret_cast<uint4*>(g.out_bf + static_cast<size_t>(row) * g.ldo + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __align__(16) __nv_bfloat16 b[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) b[i] = __float2bfloat16_rn(v[q * 8 + i]);
                o[q] = *reinterpret_cast<const uint4*>(b);
            }
        }
        if (g.out_bfT) {
#pragma unroll
            for (int i = 0; i < 32; ++i)
                g.out_bfT[static_cast<size_t>(c0 + i) * g.ldoT + row] = __float2bfloat16_rn(v[i]);
        }
    }
    if (head_w) g.head_y[row] = *g.head_b + (yacc0 + yacc);
}

// Bulk tensor store (TMA) of a shared-memory box to global memory at element
// coordinates (x, y) of the tensor map's 2-D view; completion is tracked by
// the issuing thread's bulk groups.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(src), "r"(x), "r"(y)
                 : "memory");
}

// Shared-memory staging of one epilogue warp: its 32 rows x 64 columns of the
// BF16 output (128-byte rows, the 128-byte swizzle the store's tensor map
// names: 16-byte chunk c of row r at chunk c ^ (r mod 8)), then the same block
// transposed (64 rows of 32 BF16, unswizzled).  1024-byte aligned.
constexpr int kEpiStage = 32 * 128 + 64 * 64;

// The epilogue of k_gemm_ws: the arithmetic of gemm_epilogue, the BF16 tiles
// written to shared memory and stored by TMA, one 64-column block per bulk
// group (full 128-byte lines to global memory instead of per-row pieces, and
// 64 shared-memory stores for the transposed copy instead of 32-bit-strided
// global ones).  row0: the warp's first row; lane 0 issues the stores.  The
// warp takes columns [c_lo, c_hi) (64-column blocks) and returns its part of
// the dot head: the running sums of epilogue_block added, first half + second.
template <int BN>
__device__ __forceinline__ float gemm_epilogue_tma(const GemmArgs& g, const CUtensorMap* map_out,
                                                   const CUtensorMap* map_outT, uint32_t tmem, int row0, int warp,
                                                   const float* bias, const float* head_w, unsigned char* stage,
                                                   int c_lo, int c_hi)
{
    static_assert(BN % 64 == 0, "64-column store blocks");
    const int lane = threadIdx.x & 31, row = row0 + lane;
    const uint32_t s_bf = smem_u32(stage), s_t = s_bf + 32 * 128;
    const uint32_t tl = tmem + (static_cast<uint32_t>(warp * 32) << 16);
    float yacc = 0.f, yacc0 = 0.f;
    // one half of a 64-column block into the staging tiles; the second half
    // also stores the block
    auto half_block = [&](const uint32_t (&r)[32], int c0, int half) {
        float v[32];
        epilogue_block<BN, true>(g, r, row, c0, bias, head_w, v, yacc, yacc0);
        if (half == 0) {  // the previous block's stores have read the staging tiles
            if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            __syncwarp();
        }
        if (g.out_bf) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                __nv_bfloat162 b[4];  // (round to nearest per element, as __float2bfloat16_rn)
#pragma unroll
                for (int i = 0; i < 4; ++i) b[i] = __floats2bfloat162_rn(v[q * 8 + 2 * i], v[q * 8 + 2 * i + 1]);
                const uint4 w = make_uint4(*reinterpret_cast<const uint32_t*>(&b[0]), *reinterpret_cast<const uint32_t*>(&b[1]),
                                           *reinterpret_cast<const uint32_t*>(&b[2]), *reinterpret_cast<const uint32_t*>(&b[3]));
                const uint32_t a = s_bf + lane * 128 + (((half * 4 + q) ^ (lane & 7)) << 4);
                asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w.x), "r"(w.y), "r"(w.z),
                             "r"(w.w)
                             : "memory");
            }
        }
        if (g.out_bfT) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const __nv_bfloat16 b = __float2bfloat16_rn(v[i]);
                asm volatile("st.shared.b16 [%0], %1;" ::"r"(s_t + (half * 32 + i) * 64 + lane * 2),
                             "h"(*reinterpret_cast<const unsigned short*>(&b))
                             : "memory");
            }
        }
        if (half == 1) {  // a full 64-column block: to global memory
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                if (g.out_bf) tma_store_2d(map_out, s_bf, c0 - 32, row0);
                if (g.out_bfT) tma_store_2d(map_outT, s_t, row0, c0 - 32);
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
        }
    };
    // each block's TMEM load is in flight while the block before it is worked on
    uint32_t ra[32], rb[32];
    tmem_ld32_async(tl + c_lo, ra);
    tmem_ld_wait(ra);
#pragma unroll 1
    for (int c0 = c_lo; c0 < c_hi; c0 += 64) {
        tmem_ld32_async(tl + c0 + 32, rb);
        half_block(ra, c0, 0);
        tmem_ld_wait(rb);
        if (c0 + 64 < c_hi) tmem_ld32_async(tl + c0 + 64, ra);
        half_block(rb, c0 + 32, 1);
        if (c0 + 64 < c_hi) tmem_ld_wait(ra);
    }
    return yacc0 + yacc;
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_rw(GemmArgs g)
{
    constexpr uint32_t kCols = 2 * BN;  // two accumulators of BN columns
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[kStagesRW];
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = g.K, kb = K < kKB ? K : kKB, nk = K / kb;
    unsigned char* sW = smem;                                    // nk blocks of BN x kb
    unsigned char* sA = smem + static_cast<size_t>(BN) * K * 2;  // kStagesRW stages of 128 x kb
    const int stageA = kBM * kb * 2, blockW = BN * kb * 2;
    const uint32_t sbo = (kb / 8) * 128;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStagesRW; ++i) mbar_init(smem_u32(&mbar[i]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // the weights, once (first cp.async group): block j holds B[:, j*kb .. (j+1)*kb)
    {
        const int chunks = kb / 8;
        for (int c = threadIdx.x; c < nk * BN * chunks; c += blockDim.x) {
            const int j = c / (BN * chunks), rem = c - j * BN * chunks;
            const int r = rem / chunks, kg = rem - r * chunks;
            cp_async16(smem_u32(sW + j * blockW) + (r >> 3) * sbo + (r & 7) * 16 + kg * 128,
                       g.B + static_cast<size_t>(r) * g.ldb + j * kb + kg * 8);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }

    // item i = (local tile i / nk, K block i % nk); tile t_local -> global tile
    const int tiles = g.M / kBM;
    const int bx = blockIdx.x, gx = gridDim.x;
    const int my_tiles = tiles > bx ? (tiles - 1 - bx) / gx + 1 : 0;
    const int total = my_tiles * nk;
    auto issue = [&](int item) {  // one cp.async group per item
        const int t = bx + (item / nk) * gx, j = item % nk;
        stage_tile(smem_u32(sA + (item % kStagesRW) * stageA),
                   g.A + static_cast<size_t>(t) * kBM * g.lda + j * kb, g.lda, kBM, kb);
    };
    auto epilogue = [&](int item) {  // item is the last K block of its tile
        const int tl = item / nk;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        gemm_epilogue<BN>(g, tmem + (tl & 1) * BN, (bx + tl * gx) * kBM + warp * 32 + lane, warp, g.bias,
                          g.head_w);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };
    int issued = 0;
    for (; issued < total && issued < kStagesRW; ++issued) issue(issued);
    bool ok = true;
    int waited = -1;  // every item <= waited has completed its MMAs
    for (int c = 0; c < total; ++c) {
        const int newer = issued - c - 1;  // groups committed after item c's
        if (newer >= 3)
            asm volatile("cp.async.wait_group 3;" ::: "memory");
        else if (newer == 2)
            asm volatile("cp.async.wait_group 2;" ::: "memory");
        else if (newer == 1)
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        else
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();  // also orders the previous epilogue's TMEM reads before these MMAs
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int j = c % nk;
            const uint32_t idesc = instr_desc(kBM, BN);
            const uint32_t d = tmem + ((c / nk) & 1) * BN;
            const uint32_t a0 = smem_u32(sA + (c % kStagesRW) * stageA), b0 = smem_u32(sW + j * blockW);
            for (int kk = 0; kk < kb / 16; ++kk) {
                const uint64_t da = smem_desc(a0 + kk * 256, 128, sbo);
                const uint64_t db = smem_desc(b0 + kk * 256, 128, sbo);
                const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar[c % kStagesRW]))
                : "memory");
        }
        if (c >= 1) {  // item c-1: its stage is free and, at a tile end, its accumulator final
            const int p = c - 1;
            ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[p % kStagesRW]), (p / kStagesRW) & 1));
            if (!ok) break;
            waited = p;
            if (issued < total) issue(issued++);
            if (p % nk == nk - 1) epilogue(p);
        }
    }
    if (ok && total > 0) {
        const int p = total - 1;
        ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[p % kStagesRW]), (p / kStagesRW) & 1));
        if (ok) {
            waited = p;
            epilogue(p);
        }
    }
    if (!ok && g.err && lane == 0) atomicExch(g.err, 1);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (!ok) {  // at most two committed items are unfinished; wait for them, bounded
        for (int p = waited + 1; p < total && p <= waited + 2; ++p)
            mbar_wait(smem_u32(&mbar[p % kStagesRW]), (p / kStagesRW) & 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

// ---------------------------------------------------------------- warp-specialised layer
// The same layer as k_gemm_rw (weights resident, N = BN) with the roles split
// across warps so that loading, multiplying and draining overlap:
//   warp 0     producer: the weights once, then the A tiles through kStagesWS
//              shared-memory stages.  K a multiple of 64: both by TMA into the
//              128-byte swizzled layout (the weights' boxes complete wready,
//              each A stage its full[stage]); K = 16: cp.async into core
//              matrices, waited for kLagWS groups behind, fenced into the
//              async proxy, then full[stage] signalled;
//   warp 1     one thread issues the tcgen05.mma of each K block once
//              full[stage] completes, commits to empty[stage] (the stage is
//              free again when those MMAs finish) and, at a tile's end, to
//              tfull[buf] (accumulator buffer buf = tile parity, 2 x BN TMEM
//              columns);
//   warps 2-9  the epilogue: warp w drains TMEM lanes 32 (w % 4) .. +31 of
//              buffer buf, then arrives on tempty[buf].  Eight warps (two per
//              lane quarter, half the columns each) when no transposed copy is
//              written, else warps 2-5 alone (the others have no work).
// Every wait is bounded (1 s): on a timeout the role sets *err and leaves its
// loop; the others time out in turn, and the CTA still meets at the final
// barrier before the TMEM is freed.
constexpr int kStagesWS = 4, kLagWS = 3;
constexpr int kThreadsWS = 320;

__host__ __device__ constexpr size_t gemm_ws_smem(int BN, int K)
{
    return static_cast<size_t>(BN) * K * 2 + static_cast<size_t>(kStagesWS) * kBM * (K < kKB ? K : kKB) * 2 +
           4 * kEpiStage;
}

__device__ __forceinline__ void mbar_arrive(uint32_t addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kThreadsWS, 1)
    k_gemm_ws(GemmArgs g, const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
              const __grid_constant__ CUtensorMap map_out, const __grid_constant__ CUtensorMap map_outT)
{
    constexpr uint32_t kCols = 2 * BN;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kStagesWS], empty[kStagesWS], tfull[2], tempty[2], wready;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float s_bias[BN];   // the epilogue's per-column vectors, read by every row
    __shared__ __align__(16) float s_headw[BN];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int K = g.K, kb = K < kKB ? K : kKB, nk = K / kb;
    // A tiles of 64 K columns come by TMA in the 128-byte swizzled layout (the
    // swizzle's phase is the shared address, so the block must start on 1 KB)
    const bool tma_a = kb == kKB;
    if ((smem_u32(smem) & 1023u) != 0u) {  // (uniform over the CTA: nothing allocated yet)
        if (threadIdx.x == 0 && g.err) atomicExch(g.err, 1);
        return;
    }
    unsigned char* sW = smem;
    unsigned char* sA = smem + static_cast<size_t>(BN) * K * 2;
    const int stageA = kBM * kb * 2, blockW = BN * kb * 2;
    unsigned char* sE = sA + kStagesWS * stageA;  // the epilogue warps' staging tiles
    const uint32_t sbo = (kb / 8) * 128;
    const int tiles = g.M / kBM, bx = blockIdx.x, gx = gridDim.x;
    const int my_tiles = tiles > bx ? (tiles - 1 - bx) / gx + 1 : 0;
    const int total = my_tiles * nk;
    // epilogue warps: eight (two per TMEM lane quarter, half the columns each)
    // when the second staging tile is free (no transposed copy) and the halves
    // are whole 64-column blocks, else four
    const int nepi = (g.out_bfT == nullptr && BN >= 128) ? 8 : 4;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < kStagesWS; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), nepi);
        }
        mbar_init(smem_u32(&wready), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    bool ok = true;

    if (warp == 0) {
        // ---- producer
        // the weights, resident for the CTA's tiles.  64-K blocks: one TMA box of
        // BN rows each, in the A tiles' 128-byte swizzled layout, completing on
        // wready (every CTA reads the same lines: one warp's cp.async stream of
        // them took longer than the whole main loop); else core matrices by
        // cp.async from the whole warp.
        if (tma_a) {
            if (lane == 0) {
                const uint32_t wb = smem_u32(&wready);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(wb), "r"(nk * blockW)
                             : "memory");
                for (int j = 0; j < nk; ++j) tma_load_2d(&map_b, smem_u32(sW + j * blockW), wb, j * kb, 0);
            }
        } else {
            const int chunks = kb / 8;
            for (int c = lane; c < nk * BN * chunks; c += 32) {
                const int j = c / (BN * chunks), rem = c - j * BN * chunks;
                const int r = rem / chunks, kg = rem - r * chunks;
                cp_async16(smem_u32(sW + j * blockW) + (r >> 3) * sbo + (r & 7) * 16 + kg * 128,
                           g.B + static_cast<size_t>(r) * g.ldb + j * kb + kg * 8);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        if (tma_a) {
            // one thread posts each stage's byte count on the stage's mbarrier and
            // starts its TMA copy, which completes the count (no waiting on copies
            // here)
            auto issue = [&](int i) {
                const int stage = i % kStagesWS, t = bx + (i / nk) * gx, j = i % nk;
                const uint32_t fb = smem_u32(&full[stage]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(stageA)
                             : "memory");
                tma_load_2d(&map_a, smem_u32(sA + stage * stageA), fb, j * kb, t * kBM);
            };
            const int first = total < kStagesWS ? total : kStagesWS;
            if (lane == 0) {
                for (int i = 0; i < first; ++i) issue(i);
                int issued = first;
                for (int i = first; i < total && ok; ++i) {
                    const int stage = i % kStagesWS;  // the MMAs of item i - kStagesWS released the stage
                    ok = mbar_wait(smem_u32(&empty[stage]), ((i / kStagesWS) - 1) & 1);
                    if (ok) issue(i), issued = i + 1;
                }
                // copies still in flight land before the CTA may end (each wait bounded;
                // a phase the MMA thread has already consumed answers at once)
                for (int i = issued > kStagesWS ? issued - kStagesWS : 0; i < issued; ++i)
                    if (!mbar_wait(smem_u32(&full[i % kStagesWS]), (i / kStagesWS) & 1)) ok = false;
                if (!mbar_wait(smem_u32(&wready), 0)) ok = false;
            }
            __syncwarp();
        } else {
            auto signal = [&](int item) {  // item's copies (and all older ones) are complete
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&full[item % kStagesWS]));
            };
            for (int i = 0; i < total && ok; ++i) {
                const int stage = i % kStagesWS;
                if (i >= kStagesWS)  // the MMAs of item i - kStagesWS released the stage
                    ok = mbar_wait(smem_u32(&empty[stage]), ((i / kStagesWS) - 1) & 1);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                const int t = bx + (i / nk) * gx, j = i % nk;
                const __nv_bfloat16* src = g.A + static_cast<size_t>(t) * kBM * g.lda + j * kb;
                const uint32_t dst = smem_u32(sA + stage * stageA);
                const int chunks = kb / 8;
                for (int c = lane; c < kBM * chunks; c += 32) {
                    const int r = c / chunks, kg = c - r * chunks;
                    cp_async16(dst + (r >> 3) * sbo + (r & 7) * 16 + kg * 128,
                               src + static_cast<size_t>(r) * g.lda + kg * 8);
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
                if (i >= kLagWS) {
                    asm volatile("cp.async.wait_group %0;" ::"n"(kLagWS) : "memory");
                    signal(i - kLagWS);
                }
            }
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (ok)
                for (int i = total > kLagWS ? total - kLagWS : 0; i < total; ++i) signal(i);
        }
    } else if (warp == 1) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kBM, BN);
            if (tma_a && my_tiles > 0) ok = mbar_wait(smem_u32(&wready), 0);  // the resident weights
            for (int tl = 0; tl < my_tiles && ok; ++tl) {
                const int buf = tl & 1;
                if (tl >= 2) ok = mbar_wait(smem_u32(&tempty[buf]), ((tl >> 1) - 1) & 1);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + buf * BN;
                for (int j = 0; j < nk && ok; ++j) {
                    const int i = tl * nk + j, stage = i % kStagesWS;
                    ok = mbar_wait(smem_u32(&full[stage]), (i / kStagesWS) & 1);
                    if (!ok) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = smem_u32(sA + stage * stageA), b0 = smem_u32(sW + j * blockW);
                    for (int kk = 0; kk < kb / 16; ++kk) {
                        const uint64_t da = tma_a ? smem_desc_sw128(a0 + kk * 32) : smem_desc(a0 + kk * 256, 128, sbo);
                        const uint64_t db = tma_a ? smem_desc_sw128(b0 + kk * 32) : smem_desc(b0 + kk * 256, 128, sbo);
                        const uint32_t acc = (j > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_u32(&empty[stage]))
                        : "memory");
                }
                if (!ok) break;
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&tfull[buf]))
                    : "memory");
            }
            if (ok && my_tiles > 0)  // the last accumulator is complete before the CTA may free TMEM
                ok = mbar_wait(smem_u32(&tfull[(my_tiles - 1) & 1]), ((my_tiles - 1) >> 1) & 1);
        }
        __syncwarp();
    } else if (warp - 2 < nepi) {
        // ---- epilogue warps: TMEM lanes 32 (warp % 4) + lane; with eight, warp
        // 2 + e takes the first half of the columns (e < 4) or the second,
        // staging in the quarter's second tile, and the pair adds its head parts
        // in that order (the second half's part passed through head_y: its rows
        // are the tile's own).  A warp whose wait ran out goes on through the
        // tiles without work, so that its partner never waits for it at the
        // pair's barrier.
        const int q = warp & 3, h = (warp - 2) >> 2, cw = BN * 4 / nepi;
        const bool pair_head = g.head_w && nepi == 8;
        // the per-column vectors, read only here: loaded by these warps while the
        // first copies and MMAs go on (not before the CTA's opening barrier)
        for (int n = threadIdx.x - 64; n < BN; n += nepi * 32) {
            s_bias[n] = g.bias ? g.bias[n] : 0.f;
            s_headw[n] = g.head_w ? g.head_w[n] : 0.f;
        }
        asm volatile("bar.sync 5, %0;" ::"r"(nepi * 32) : "memory");
        for (int tl = 0; tl < my_tiles; ++tl) {
            const int buf = tl & 1, row0 = (bx + tl * gx) * kBM + q * 32;
            float part = 0.f;
            if (ok) ok = mbar_wait(smem_u32(&tfull[buf]), (tl >> 1) & 1);
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                part = gemm_epilogue_tma<BN>(g, &map_out, &map_outT, tmem + buf * BN, row0, q,
                                             g.bias ? s_bias : nullptr, g.head_w ? s_headw : nullptr,
                                             sE + q * kEpiStage + h * (32 * 128), h * cw, h * cw + cw);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
            }
            if (pair_head) {
                if (h == 1) g.head_y[row0 + lane] = part;
                asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");
                if (h == 0) g.head_y[row0 + lane] = *g.head_b + (part + g.head_y[row0 + lane]);
            } else if (g.head_w && ok) {
                g.head_y[row0 + lane] = *g.head_b + part;
            }
            if (ok && lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
        }
        if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the stores are done
        __syncwarp();
    }
    if (!ok && g.err && lane == 0) atomicExch(g.err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols)
                     : "memory");
}

// Failure-path check of the bounded waits: one CTA takes TMEM and waits, with
// the same routine as every tensor-core kernel above, on an mbarrier that no
// copy or MMA will ever complete.  The wait gives up after limit_ns; the CTA
// then sets *err (as the real kernels do), frees its TMEM and ends, so the
// context stays usable.  Nothing here faults or hangs.
__global__ void __launch_bounds__(kThreads, 1) k_wait_probe(int* err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(32)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&mbar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const bool ok = __syncthreads_and(mbar_wait_for(smem_u32(&mbar), 0u, limit_ns));
    if (!ok && err && threadIdx.x == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32) : "memory");
    (void)lane;
}

// ---------------------------------------------------------------- the whole network on one tile
// The three layers of a network on one 128-row tile with the activations kept
// on chip.  The layer-1 inputs sit in a small shared-memory tile; each later
// layer's BF16 inputs in one activation tile (128 rows x up to 256 columns, in
// 32-column blocks of the core-matrix layout); the FP32 accumulators in two
// 256-column TMEM regions that the layers alternate between.  The weights
// stream from global memory (L2) through a ring of four shared-memory buffers,
// one 32-column block per bulk asynchronous copy (cp.async.bulk, completion
// counted in bytes on an mbarrier), each block already packed in the layout
// the MMA descriptors read.
//
// Roles (warp-specialised, no CTA-wide barrier inside a tile):
//   epilogue warps (kEpi = 4 or 8; warp w drains TMEM lane quarter w % 4, and
//     with 8 warps half the columns of each block): wait for a layer's
//     accumulator (mbarrier `done`), then write the next layer's inputs one
//     32-column block at a time (bias, ReLU, BF16), announcing each block on
//     its own mbarrier a[j]; after layer 3 the head (bias, ReLU, linear output).
//   one MMA-issuing thread (lane 0 of warp kEpi): issues each block's MMAs as
//     soon as its inputs are announced and its weights have landed, so the
//     tensor core works while the epilogue goes on;
//   one loading thread (lane 0 of warp kEpi + 1): starts each weight block's
//     copy as soon as the buffer it reuses has been released by the MMAs.
// The MMA sequence (K steps of 16 in column order) and the epilogue arithmetic
// are those of k_gemm_ws, so a tile computes bitwise what the layer-by-layer
// kernels compute.

// Packed BF16 weights and FP32 vectors of one network.  Blocks, each contiguous:
//   w1p  W1, h1 x 16, core-matrix layout with 8-row groups 256 bytes apart
//   w2p  h1 / 32 blocks, block j = W2[:, 32 j .. 32 j + 31] (h2 x 32, groups 512 bytes apart)
//   w3p  h2 / 32 blocks of W3 (h3 x 32)
struct MlpView {
    const __nv_bfloat16* w1p;
    const __nv_bfloat16* w2p;
    const __nv_bfloat16* w3p;
    const float* b2;
    const float* b3;
    const float* w4;
    const float* b4;
    int enc, h1, h2, h3;
    int* err;  // set to 1 when a wait runs out
};

constexpr int kRingDepth = 4;                  // weight buffers
constexpr int kBlockK = 32;                    // input columns per weight block of layers 2 and 3
constexpr int kMaxBlocks = 256 / kBlockK;      // activation blocks
constexpr int kTileRing = 256 * kBlockK * 2;   // one staged weight block (at most 256 x 32 BF16)
constexpr int kTileA1 = kBM * 16 * 2;          // layer-1 inputs
constexpr int kTileSub = kBM * kBlockK * 2;    // one 32-column block of the activations
constexpr int kTileA = kBM * 256 * 2;          // the activation tile
constexpr int kTileVec = 3 * 256 * 4 + 2 * kBM * 4;  // b2, b3, w4; the head's two partial sums per row
// the engine's shared memory: ring | layer-1 inputs | activations | vectors | head partials
constexpr int kOffA1 = kRingDepth * kTileRing;
constexpr int kOffA = kOffA1 + kTileA1;
constexpr int kOffVec = kOffA + kTileA;
constexpr size_t kTileSmem = kOffVec + kTileVec;
// mbarriers: full[kRingDepth], empty[kRingDepth], done, a1, a[kMaxBlocks]
constexpr int kTileBars = 2 * kRingDepth + 2 + kMaxBlocks;
constexpr uint32_t kTileCols = 512;            // two accumulators

// Threads of a CTA running the engine with kEpi epilogue warps: those, then the
// MMA-issuing warp (warp kEpi), then the weight-loading warp (warp kEpi + 1);
// one thread of each of the last two does the work.
__host__ __device__ constexpr int tile_threads(int kEpi) { return (kEpi + 2) * 32; }

__host__ __device__ inline int mlp_blocks(const MlpView& v) { return 1 + v.h1 / kBlockK + v.h2 / kBlockK; }

// Start the bulk copy of block b of the network (0 = W1, then W2's, then W3's)
// into the ring buffer at dst, completing on full_bar.  One thread.
__device__ __forceinline__ void mlp_issue_block(const MlpView& v, int b, uint32_t dst, uint32_t full_bar)
{
    const int n2 = v.h1 / kBlockK;
    const __nv_bfloat16* src;
    uint32_t bytes;
    if (b == 0) {
        src = v.w1p;
        bytes = static_cast<uint32_t>(v.h1) * 16 * 2;
    } else if (b <= n2) {
        src = v.w2p + static_cast<size_t>(b - 1) * v.h2 * kBlockK;
        bytes = static_cast<uint32_t>(v.h2) * kBlockK * 2;
    } else {
        src = v.w3p + static_cast<size_t>(b - 1 - n2) * v.h3 * kBlockK;
        bytes = static_cast<uint32_t>(v.h3) * kBlockK * 2;
    }
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(full_bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(full_bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_cta(uint32_t addr)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

// Pipeline state of one CTA's tiles.  Weight blocks are numbered across tiles:
// block g lives in ring buffer g % kRingDepth and completes phase
// (g / kRingDepth) & 1 of full[that buffer] (landed) and of empty[that buffer]
// (its MMAs done).  Barrier addresses are computed, not indexed, so that the
// state stays in registers.  next / apar / tiles belong to the MMA-issuing
// thread, issued to the loading thread, layers (phases of `done`) to the
// epilogue threads.
struct MlpTiles {
    uint32_t ring, sA1, sA;  // shared addresses
    uint32_t bars;           // the mbarriers, 8 bytes apart in the order above
    uint32_t tmem;           // kTileCols columns
    int next;                // next weight block to multiply
    int issued;              // blocks whose copy has been started
    int total;               // blocks this CTA will multiply in all
    int layers;              // layers completed
    uint32_t apar;           // bit j: parity of a[j]'s next phase
    int tiles;               // tiles issued
};

__device__ __forceinline__ uint32_t tile_full(const MlpTiles& t, int b) { return t.bars + 8 * b; }
__device__ __forceinline__ uint32_t tile_empty(const MlpTiles& t, int b) { return t.bars + 8 * (kRingDepth + b); }
__device__ __forceinline__ uint32_t tile_done(const MlpTiles& t) { return t.bars + 8 * (2 * kRingDepth); }
__device__ __forceinline__ uint32_t tile_a1(const MlpTiles& t) { return t.bars + 8 * (2 * kRingDepth + 1); }
__device__ __forceinline__ uint32_t tile_a(const MlpTiles& t, int j) { return t.bars + 8 * (2 * kRingDepth + 2 + j); }
// Tile k's accumulator for layers 1 and 3 (which = 0) or for layer 2 (which = 1):
// the two 256-column regions, their roles swapped on odd tiles.
__device__ __forceinline__ uint32_t tile_acc(const MlpTiles& t, int k, int which)
{
    return t.tmem + (((k ^ which) & 1) ? 256u : 0u);
}

// Every thread of the CTA: addresses, then (warp 0) the TMEM columns and (the
// MMA-issuing thread) the barriers.  The caller then runs the TMEM-allocation
// fence / barrier / fence sequence, reads *tmem_slot, and has the loading thread
// run mlp_load_all.
template <int kEpi>
__device__ __forceinline__ void mlp_tiles_init(MlpTiles& t, const MlpView& v, uint32_t smem_base, uint64_t* bars,
                                               uint32_t* tmem_slot, int total)
{
    t.ring = smem_base;
    t.sA1 = smem_base + kOffA1;
    t.sA = smem_base + kOffA;
    t.bars = smem_u32(bars);
    t.tmem = 0;
    t.next = t.issued = t.layers = t.tiles = 0;
    t.apar = 0u;
    t.total = total;
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTileCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == kEpi * 32) {
        for (int b = 0; b < 2 * kRingDepth + 1; ++b) mbar_init(t.bars + 8 * b, 1);  // ring, done: one arrival
        mbar_init(tile_a1(t), kBM / 32);                                             // the four encoding warps
        for (int j = 0; j < kMaxBlocks; ++j) mbar_init(tile_a(t, j), kEpi);         // every epilogue warp
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
}

// The loading thread: the copies of the weight blocks this CTA will multiply
// (those before block `upto`), in order, each as soon as the ring buffer it
// reuses is free (the MMAs of the block kRingDepth before it are done).  False
// when a wait ran out.
__device__ __forceinline__ bool mlp_load_all(const MlpView& v, MlpTiles& t, int upto = 1 << 30)
{
    const int nb = mlp_blocks(v);
    for (; t.issued < t.total && t.issued < upto; ++t.issued) {
        const int b = t.issued % kRingDepth;
        if (t.issued >= kRingDepth && !mbar_wait(tile_empty(t, b), ((t.issued / kRingDepth) - 1) & 1)) return false;
        mlp_issue_block(v, t.issued % nb, t.ring + b * kTileRing, tile_full(t, b));
    }
    return true;
}

// The issuing thread: the MMAs of the next weight block (A block at a0 with
// 8-row groups sbo_a bytes apart, kb input columns) into accumulator d, once
// its weights have landed, committed to the block's empty barrier (which
// frees its buffer for the loading thread).  False when a wait ran out.
__device__ __forceinline__ bool mlp_mma_block(const MlpView& v, MlpTiles& t, uint32_t a0, uint32_t sbo_a, int kb,
                                              uint32_t d, uint32_t idesc, bool first)
{
    const int g = t.next, buf = g % kRingDepth;
    if (!mbar_wait(tile_full(t, buf), (g / kRingDepth) & 1)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t b0 = t.ring + buf * kTileRing, sbo_b = (kb / 8) * 128;
    for (int kk = 0; kk < kb / 16; ++kk) {
        const uint64_t da = smem_desc(a0 + kk * 256, 128, sbo_a);
        const uint64_t db = smem_desc(b0 + kk * 256, 128, sbo_b);
        const uint32_t acc = (!first || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tile_empty(t, buf))
                 : "memory");
    ++t.next;
    return true;
}

__device__ __forceinline__ void mlp_commit_done(const MlpTiles& t)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tile_done(t))
                 : "memory");
}

// The issuing thread's part of one tile: layer 1 once the encoding warps have
// announced the inputs, then each block of layers 2 and 3 once the epilogue
// warps have announced it, each layer committed to `done`.  False when a wait
// ran out (the epilogue warps then time out on `done`).
__device__ __forceinline__ bool mlp_tile_issue(const MlpView& v, MlpTiles& t)
{
    // the two accumulators swap roles from tile to tile: layer 1 of a tile goes
    // where the tile before kept layer 2, free once its epilogue has announced
    // all of layer 2's blocks (which this thread waited for before the last
    // layer-3 MMAs), so it need not wait for that tile's head
    const uint32_t RA = tile_acc(t, t.tiles, 0), RB = tile_acc(t, t.tiles, 1);  // layers 1 and 3 | layer 2
    if (!mbar_wait(tile_a1(t), t.tiles & 1)) return false;
    ++t.tiles;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!mlp_mma_block(v, t, t.sA1, 256, 16, RA, instr_desc(kBM, v.h1), true)) return false;
    mlp_commit_done(t);
    for (int L = 2; L <= 3; ++L) {
        const int K = L == 2 ? v.h1 : v.h2, N = L == 2 ? v.h2 : v.h3;
        const uint32_t idesc = instr_desc(kBM, N);
        for (int j = 0; j < K / kBlockK; ++j) {
            if (!mbar_wait(tile_a(t, j), (t.apar >> j) & 1u)) return false;
            t.apar ^= 1u << j;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!mlp_mma_block(v, t, t.sA + j * kTileSub, kTileSub / 16, kBlockK, L == 2 ? RB : RA, idesc, j == 0))
                return false;
        }
        mlp_commit_done(t);
    }
    return true;
}

// TMEM -> registers, 16 consecutive FP32 columns of this thread's lane, without
// the wait: the registers are valid after tmem_ld16_wait on them (which waits
// for every load this thread has issued).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16_wait(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])::"memory");
}

// One thread's 16 columns of one row of a 32-column activation block, from the
// accumulator values r: + bias (nullable; 16-byte aligned shared memory), ReLU,
// BF16, as two 8-column core-matrix rows at dst (the second 128 bytes after the
// first).
__device__ __forceinline__ void mlp_act_regs(const uint32_t (&r)[16], const float* bias, uint32_t dst)
{
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float b[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (bias) {
            const float4 lo = lds4(bias + q * 8), hi = lds4(bias + q * 8 + 4);
            b[0] = lo.x, b[1] = lo.y, b[2] = lo.z, b[3] = lo.w, b[4] = hi.x, b[5] = hi.y, b[6] = hi.z, b[7] = hi.w;
        }
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float x0 = __uint_as_float(r[q * 8 + 2 * i]), x1 = __uint_as_float(r[q * 8 + 2 * i + 1]);
            if (bias) {
                x0 += b[2 * i];
                x1 += b[2 * i + 1];
            }
            x0 = fmaxf(x0, 0.f);
            x1 = fmaxf(x1, 0.f);
            const __nv_bfloat162 p = __floats2bfloat162_rn(x0, x1);  // (x0 in the low half)
            w[i] = *reinterpret_cast<const uint32_t*>(&p);
        }
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst + q * 128), "r"(w[0]), "r"(w[1]),
                     "r"(w[2]), "r"(w[3])
                     : "memory");
    }
}

// Every epilogue thread: wait until the layer the issuing thread committed to
// `done` has completed.  False (on this thread) when the wait ran out.
__device__ __forceinline__ bool mlp_wait_layer(MlpTiles& t)
{
    const bool ok = mbar_wait(tile_done(t), t.layers & 1);
    ++t.layers;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return ok;
}

// Announce an activation block (or the layer-1 inputs) to the issuing thread:
// this warp's generic shared-memory writes made visible to the tensor core's
// async proxy, its TMEM reads ordered before the MMAs that follow, one arrival
// per warp.
__device__ __forceinline__ void mlp_announce(uint32_t bar)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive_cta(bar);
}

// The epilogue warps' part of one tile, after the encoding warps (0-3) have
// written the layer-1 inputs to t.sA1 and announced them on a1: layers 1 and 2's
// outputs into the activation blocks, then the head.  Warp w drains TMEM lane
// quarter w % 4 (row = 32 (w % 4) + lane); with 8 warps, half w / 4 of each
// block's columns.  The head sums each half of layer 3's columns in column
// order and adds the halves; rows 0..127 get their output in *y (threads
// 0..127).  bar_id: a named barrier free for the kEpi warps (8 warps only).
// False (on every epilogue thread) when a wait ran out.
// after_e1 / after_e2: called on every epilogue thread once layer 1's / layer
// 2's outputs are all stored, while the tensor core finishes the layer after
// them (a window in which the epilogue warps would only wait).
template <int kEpi, typename AfterE1, typename AfterE2>
__device__ __forceinline__ bool mlp_tile_epilogue(const MlpView& v, MlpTiles& t, const float* s_b2, const float* s_b3,
                                                  const float* s_w4, float* s_part, float b4, float* y,
                                                  AfterE1&& after_e1, AfterE2&& after_e2)
{
    static_assert(kEpi == 4 || kEpi == 8, "four or eight epilogue warps");
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, row = quarter * 32 + lane;
    const uint32_t lane_off = static_cast<uint32_t>(quarter * 32) << 16;
    const int tk = t.layers / 3;  // this tile's index among the CTA's tiles
    const uint32_t RA = tile_acc(t, tk, 0), RB = tile_acc(t, tk, 1);  // layers 1 and 3 | layer 2
    bool ok = mlp_wait_layer(t);  // layer 1
    // the warp's 16-column pieces of a layer in order: piece u is half hf of
    // block u / H (with 8 warps one half, warp / 4, of every block); each piece's
    // TMEM load is in flight while the piece before it is worked on, and a
    // block is announced once its last piece is stored
    constexpr int H = kEpi == 8 ? 1 : 2;
    for (int L = 2; L <= 3 && ok; ++L) {
        const int K = L == 2 ? v.h1 : v.h2, nu = (K / kBlockK) * H;
        const uint32_t src = (L == 2 ? RA : RB) + lane_off;
        const float* bias = L == 2 ? nullptr : s_b2;
        auto col = [&](int u) { return (u / H) * kBlockK + 16 * (kEpi == 8 ? (warp >> 2) : (u % H)); };
        auto piece = [&](const uint32_t (&r)[16], int u) {
            const int c = col(u), j = u / H, hf = (c % kBlockK) / 16;
            mlp_act_regs(r, bias ? bias + c : nullptr,
                         t.sA + j * kTileSub + (row >> 3) * (kTileSub / 16) + (row & 7) * 16 + (2 * hf) * 128);
            if (u % H == H - 1) mlp_announce(tile_a(t, j));
        };
        uint32_t ra[16], rb[16];
        tmem_ld16_async(src + col(0), ra);
        tmem_ld16_wait(ra);
#pragma unroll 1
        for (int u = 0; u < nu; u += 2) {
            if (u + 1 < nu) tmem_ld16_async(src + col(u + 1), rb);
            piece(ra, u);
            if (u + 1 < nu) {
                tmem_ld16_wait(rb);
                if (u + 2 < nu) tmem_ld16_async(src + col(u + 2), ra);
                piece(rb, u + 1);
                if (u + 2 < nu) tmem_ld16_wait(ra);
            }
        }
        if (L == 2)
            after_e1();
        else
            after_e2();
        ok = mlp_wait_layer(t);  // layer L
    }
    // head: each half of layer 3's columns in column order, then the halves added
    const int hh = v.h3 / 2;
    float part[2] = {0.f, 0.f};
    if (ok) {
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
            if (kEpi == 8 && hf != (warp >> 2)) continue;
            float yacc = 0.f;
            auto acc16 = [&](const uint32_t (&r)[16], int c0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 bq = lds4(s_b3 + c0 + 4 * q), wq = lds4(s_w4 + c0 + 4 * q);
                    const float bb[4] = {bq.x, bq.y, bq.z, bq.w}, ww[4] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float x = fmaxf(__uint_as_float(r[4 * q + i]) + bb[i], 0.f);
                        yacc = fmaf(ww[i], x, yacc);
                    }
                }
            };
            // the columns of this half in order, 16 at a time, the next load in flight
            const int c_lo = hf * hh, c_hi = c_lo + hh;
            uint32_t ra[16], rb[16];
            tmem_ld16_async(RA + lane_off + c_lo, ra);
            tmem_ld16_wait(ra);
#pragma unroll 1
            for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
                if (c0 + 16 < c_hi) tmem_ld16_async(RA + lane_off + c0 + 16, rb);
                acc16(ra, c0);
                if (c0 + 16 < c_hi) {
                    tmem_ld16_wait(rb);
                    if (c0 + 32 < c_hi) tmem_ld16_async(RA + lane_off + c0 + 32, ra);
                    acc16(rb, c0 + 16);
                    if (c0 + 32 < c_hi) tmem_ld16_wait(ra);
                }
            }
            part[hf] = yacc;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");  // these TMEM reads before the next tile's MMAs
    if (kEpi == 8) {
        if (warp >= 4) s_part[row] = part[1];
        asm volatile("bar.sync 1, %0;" ::"n"(kEpi * 32) : "memory");
        if (warp < 4) part[1] = s_part[row];
        asm volatile("bar.sync 1, %0;" ::"n"(kEpi * 32) : "memory");  // s_part free again
    }
    if (tid < kBM) *y = b4 + (part[0] + part[1]);
    return ok;
}

template <int kEpi>
__device__ __forceinline__ bool mlp_tile_epilogue(const MlpView& v, MlpTiles& t, const float* s_b2, const float* s_b3,
                                                  const float* s_w4, float* s_part, float b4, float* y)
{
    return mlp_tile_epilogue<kEpi>(v, t, s_b2, s_b3, s_w4, s_part, b4, y, [] {}, [] {});
}

// AND of v over the `threads` threads meeting at named barrier `id`.
__device__ __forceinline__ bool bar_and(int id, int threads, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, %2, %3, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(v)), "r"(id), "r"(threads)
        : "memory");
    return r != 0;
}

// After a failure: the loading thread waits (bounded) for the copies it started
// and the MMA-issuing thread for its last MMAs, so that nothing writes this
// CTA's shared memory or TMEM once it moves on.  Each waits on its own state.
__device__ __forceinline__ void mlp_drain_loads(MlpTiles& t)
{
    for (int g = t.issued - kRingDepth > 0 ? t.issued - kRingDepth : 0; g < t.issued; ++g)
        mbar_wait(tile_full(t, g % kRingDepth), (g / kRingDepth) & 1);
}

__device__ __forceinline__ void mlp_drain_mmas(MlpTiles& t)
{
    if (t.next > 0) {
        const int g = t.next - 1;
        mbar_wait(tile_empty(t, g % kRingDepth), (g / kRingDepth) & 1);
    }
}

}  // namespace tc

// ---------------------------------------------------------------- MLP helpers

constexpr int kMlpIn = 16, kMlpHid = 256;  // input width; widest hidden layer
constexpr int kSplitMax = 74;  // split-K of a weight gradient: 2 x 74 CTAs cover the 148 SMs
constexpr int kMlpParams = kMlpHid * kMlpIn + 2 * (kMlpHid * kMlpHid + kMlpHid) + kMlpHid + 1;

// Surrogate network x (16) -> h1 -> h2 -> h3 -> 1 (ReLU hidden, linear output,
// no first-layer bias: the encoding carries a constant one).  Flat FP32
// parameters W1 (h1 x 16) | W2 (h2 x h1) | b2 | W3 (h3 x h2) | b3 | w4 | b4.
// Encodings: 0 x_j = theta_j / 3, x_7 = 1; 1 (jointNERF, Sec. 4.2)
// x_j = sin theta_j, x_{7+j} = cos theta_j, x_14 = 1.
struct MlpArch {
    int enc, h1, h2, h3;
    int oW1, oW2, ob2, oW3, ob3, ow4, ob4, count;
};

__host__ __device__ inline MlpArch mlp_arch(int enc, int h1, int h2, int h3)
{
    MlpArch a{enc, h1, h2, h3, 0, 0, 0, 0, 0, 0, 0, 0};
    a.oW1 = 0;
    a.oW2 = a.oW1 + h1 * kMlpIn;
    a.ob2 = a.oW2 + h2 * h1;
    a.oW3 = a.ob2 + h2;
    a.ob3 = a.oW3 + h3 * h2;
    a.ow4 = a.ob3 + h3;
    a.ob4 = a.ow4 + h3;
    a.count = a.ob4 + 1;
    return a;
}

// The encoded inputs of one configuration theta (dof <= 7 joints).
__device__ __forceinline__ void mlp_encode_row(const float* th, int dof, int enc, float (&v)[kMlpIn])
{
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) v[i] = 0.f;
    if (enc == 1) {
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            if (j < dof) {
                float sj, cj;
                sincosf(th[j], &sj, &cj);
                v[j] = sj;
                v[7 + j] = cj;
            }
        }
        v[14] = 1.f;
    } else {
#pragma unroll
        for (int j = 0; j < 7; ++j)
            if (j < dof) v[j] = th[j] / 3.f;
        v[7] = 1.f;
    }
}

// Inputs of the encoding; rows count..rows_pad-1 are zero.
// x: rows_pad x 16; xT (nullable): 16 x rows_pad.
__global__ void k_mlp_encode(const float* __restrict__ theta, int count, int dof, int rows_pad, int enc,
                             __nv_bfloat16* __restrict__ x, __nv_bfloat16* __restrict__ xT)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows_pad) return;
    float v[kMlpIn];
    if (r < count) {
        mlp_encode_row(theta + static_cast<size_t>(r) * dof, dof, enc, v);
    } else {
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < kMlpIn; ++i) {
        const __nv_bfloat16 b = __float2bfloat16_rn(v[i]);
        x[static_cast<size_t>(r) * kMlpIn + i] = b;
        if (xT) xT[static_cast<size_t>(i) * rows_pad + r] = b;
    }
}

// Row `row` (0..127) of a tile's layer-1 inputs (128 x 16 BF16, 8-row groups 256
// bytes apart, the two 8-column halves 128 bytes apart) from encoded values v.
__device__ __forceinline__ void mlp_store_input_row(uint32_t sA, int row, const float (&v)[kMlpIn])
{
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat16 b0 = __float2bfloat16_rn(v[2 * i]), b1 = __float2bfloat16_rn(v[2 * i + 1]);
        w[i] = static_cast<uint32_t>(__bfloat16_as_ushort(b0)) | (static_cast<uint32_t>(__bfloat16_as_ushort(b1)) << 16);
    }
    const uint32_t a = sA + (row >> 3) * 256 + (row & 7) * 16;
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3])
                 : "memory");
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a + 128), "r"(w[4]), "r"(w[5]), "r"(w[6]),
                 "r"(w[7])
                 : "memory");
}

// BF16 weights (row-major, out x in) -> the packed blocks of tc::MlpView.
__global__ void k_mlp_pack(const __nv_bfloat16* __restrict__ w1, const __nv_bfloat16* __restrict__ w2,
                           const __nv_bfloat16* __restrict__ w3, int h1, int h2, int h3,
                           __nv_bfloat16* __restrict__ w1p, __nv_bfloat16* __restrict__ w2p,
                           __nv_bfloat16* __restrict__ w3p)
{
    constexpr int KB = tc::kBlockK;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < h1 * kMlpIn) {  // (n, k): 8-row groups of 128 elements, rows of 8, two halves of K
        const int n = i / kMlpIn, k = i - n * kMlpIn;
        w1p[(n >> 3) * 128 + (n & 7) * 8 + (k >> 3) * 64 + (k & 7)] = w1[i];
    }
    if (i < h2 * h1) {  // block k / 32: h2 x 32, 8-row groups of 256 elements
        const int n = i / h1, k = i - n * h1, kk = k % KB;
        w2p[static_cast<size_t>(k / KB) * h2 * KB + (n >> 3) * (8 * KB) + (n & 7) * 8 + (kk >> 3) * 64 + (kk & 7)] = w2[i];
    }
    if (i < h3 * h2) {
        const int n = i / h2, k = i - n * h2, kk = k % KB;
        w3p[static_cast<size_t>(k / KB) * h3 * KB + (n >> 3) * (8 * KB) + (n & 7) * 8 + (kk >> 3) * 64 + (kk & 7)] = w3[i];
    }
}

// Inference on count configurations with the whole network per 128-row tile
// (tc::mlp_tile_*): one persistent CTA per SM walks the tiles with eight
// epilogue warps and one issuing warp; the rows' encoded inputs go straight
// from theta into shared memory, and nothing but y is written.  y gets rows
// 0..count-1.  Bitwise what mlp_forward computes.
constexpr int kFwdEpi = 8;

__global__ void __launch_bounds__(tc::tile_threads(kFwdEpi), 1)
k_mlp_forward_tiles(tc::MlpView v, const float* __restrict__ theta, int count, int dof, float* __restrict__ y)
{
    extern __shared__ __align__(16) unsigned char tile_smem[];
    __shared__ __align__(8) uint64_t bars[tc::kTileBars];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles = (count + tc::kBM - 1) / tc::kBM;
    const int my_tiles = tiles > static_cast<int>(blockIdx.x) ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    float* s_b2 = reinterpret_cast<float*>(tile_smem + tc::kOffVec);
    float* s_b3 = s_b2 + 256;
    float* s_w4 = s_b3 + 256;
    float* s_part = s_w4 + 256;
    tc::MlpTiles t;
    tc::mlp_tiles_init<kFwdEpi>(t, v, tc::smem_u32(tile_smem), bars, &tmem_slot, my_tiles * tc::mlp_blocks(v));
    for (int n = tid; n < 256; n += blockDim.x) {
        s_b2[n] = n < v.h2 ? v.b2[n] : 0.f;
        s_b3[n] = n < v.h3 ? v.b3[n] : 0.f;
        s_w4[n] = n < v.h3 ? v.w4[n] : 0.f;
    }
    const float b4 = *v.b4;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    t.tmem = tmem_slot;
    bool ok = true;
    if (warp == kFwdEpi + 1) {  // the loading warp: one thread
        if ((tid & 31) == 0 && !tc::mlp_load_all(v, t)) {
            if (v.err) atomicExch(v.err, 1);
            tc::mlp_drain_loads(t);
        }
    } else if (warp == kFwdEpi) {  // the MMA-issuing warp: one thread
        if ((tid & 31) == 0) {
            for (int k = 0; k < my_tiles && ok; ++k) ok = tc::mlp_tile_issue(v, t);
            if (!ok) {
                if (v.err) atomicExch(v.err, 1);
                tc::mlp_drain_mmas(t);
            }
        }
    } else {
        // The four encoding warps (threads 0..127, one row each) write a tile's
        // layer-1 inputs.  Tile k + 1's are loaded once tile k's layer-1 outputs
        // are stored and encoded once its layer-2 outputs are, while the tensor
        // core finishes the next layer (its layer 1 has long read them).
        float thr[7];
        auto load_row = [&](int k) {
            const int row = (blockIdx.x + k * gridDim.x) * tc::kBM + tid;
#pragma unroll
            for (int j = 0; j < 7; ++j) thr[j] = (row < count && j < dof) ? theta[static_cast<size_t>(row) * dof + j] : 0.f;
        };
        auto encode_row = [&](int k) {
            const int row = (blockIdx.x + k * gridDim.x) * tc::kBM + tid;
            float in[kMlpIn];
            if (row < count) {
                mlp_encode_row(thr, dof, v.enc, in);
            } else {
#pragma unroll
                for (int i = 0; i < kMlpIn; ++i) in[i] = 0.f;
            }
            mlp_store_input_row(t.sA1, tid, in);
            tc::mlp_announce(tc::tile_a1(t));
        };
        if (tid < tc::kBM && my_tiles > 0) {
            load_row(0);
            encode_row(0);
        }
        for (int k = 0; k < my_tiles && ok; ++k) {
            const int row = (blockIdx.x + k * gridDim.x) * tc::kBM + tid;  // threads 0..127
            const bool next = tid < tc::kBM && k + 1 < my_tiles;
            float out = 0.f;
            ok = tc::mlp_tile_epilogue<kFwdEpi>(v, t, s_b2, s_b3, s_w4, s_part, b4, &out,
                                                [&] { if (next) load_row(k + 1); },
                                                [&] { if (next) encode_row(k + 1); });
            ok = tc::bar_and(2, kFwdEpi * 32, ok);  // the same decision on every epilogue thread
            if (ok && tid < tc::kBM && row < count) y[row] = out;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(t.tmem), "r"(tc::kTileCols) : "memory");
}

// FP32 master weights -> BF16 operands: W1, W2, W3 and the transposes W2^T (h1 x h2), W3^T (h2 x h3).
__global__ void k_mlp_cast(const float* __restrict__ p, MlpArch A, __nv_bfloat16* __restrict__ w1,
                           __nv_bfloat16* __restrict__ w2, __nv_bfloat16* __restrict__ w2t,
                           __nv_bfloat16* __restrict__ w3, __nv_bfloat16* __restrict__ w3t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < A.h1 * kMlpIn) w1[i] = __float2bfloat16_rn(p[A.oW1 + i]);
    if (i < A.h2 * A.h1) {
        const int n = i / A.h1, k = i - n * A.h1;
        const __nv_bfloat16 a = __float2bfloat16_rn(p[A.oW2 + i]);
        w2[i] = a;
        w2t[k * A.h2 + n] = a;
    }
    if (i < A.h3 * A.h2) {
        const int n = i / A.h2, k = i - n * A.h2;
        const __nv_bfloat16 b = __float2bfloat16_rn(p[A.oW3 + i]);
        w3[i] = b;
        w3t[k * A.h3 + n] = b;
    }
}

// He-uniform initialisation from the Philox stream (tag 1): W ~ U(-sqrt(6/fan_in),
// sqrt(6/fan_in)) with fan_in the number of encoded features + 1 for the first
// layer (whose bias column and padding start at 0), biases 0.
__global__ void k_mlp_init(float* __restrict__ p, MlpArch A, uint32_t seed_lo, uint32_t seed_hi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.count) return;
    const uint4 r = storm::philox4x32_10(make_uint4(static_cast<uint32_t>(i), 0u, 0u, 1u), seed_lo, seed_hi);
    const float u = 2.f * storm::bits_to_unit(r.x) - 1.f;
    const int feats = A.enc == 1 ? 14 : 7;
    float v = 0.f;
    if (i < A.oW2) {
        v = (i % kMlpIn) < feats ? u * sqrtf(6.f / static_cast<float>(feats + 1)) : 0.f;
    } else if (i < A.ob2) {
        v = u * sqrtf(6.f / static_cast<float>(A.h1));
    } else if (i >= A.oW3 && i < A.ob3) {
        v = u * sqrtf(6.f / static_cast<float>(A.h2));
    } else if (i >= A.ow4 && i < A.ob4) {
        v = u * sqrtf(6.f / static_cast<float>(A.h3));
    }
    p[i] = v;
}

// Output layer gradient of the mean squared error: r = y - t, dy = 2 r / count,
// delta3 = dy w4 o [a3 > 0] (BF16, row-major and transposed); rows >= count get 0.
// One block of h3 threads per row; loss_part[row] = r^2.
__global__ void __launch_bounds__(256)
k_mlp_dhead(const float* __restrict__ y, const float* __restrict__ t, int count, int rows_pad, MlpArch A,
            const __nv_bfloat16* __restrict__ a3, const float* __restrict__ p,
            float* __restrict__ dy, __nv_bfloat16* __restrict__ d3, __nv_bfloat16* __restrict__ d3T,
            float* __restrict__ loss_part)
{
    const int b = blockIdx.x, n = threadIdx.x;
    const float r = (b < count) ? y[b] - t[b] : 0.f;
    const float g = 2.f * r / static_cast<float>(count);
    if (n == 0) dy[b] = g;
    const float a = __bfloat162float(a3[static_cast<size_t>(b) * A.h3 + n]);
    const __nv_bfloat16 v = __float2bfloat16_rn(a > 0.f ? g * p[A.ow4 + n] : 0.f);
    d3[static_cast<size_t>(b) * A.h3 + n] = v;
    d3T[static_cast<size_t>(n) * rows_pad + b] = v;
    if (n == 0) loss_part[b] = r * r;
}

// out[n] = sum_b rows[n][b] (rows: n x rows_pad, contiguous), one block per n.
__global__ void __launch_bounds__(256)
k_mlp_rowsum(const __nv_bfloat16* __restrict__ rows, int rows_pad, float* __restrict__ out)
{
    __shared__ float sh[32];
    const int n = blockIdx.x;
    float acc = 0.f;
    for (int b = threadIdx.x; b < rows_pad; b += blockDim.x)
        acc += __bfloat162float(rows[static_cast<size_t>(n) * rows_pad + b]);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[n] = acc;
}

// dw4[n] = sum_b dy_b a3[b][n]; db4 = sum_b dy_b; loss = sum_b r_b^2 / count.
// Grid h3 + 2.
__global__ void __launch_bounds__(256)
k_mlp_head_grad(const float* __restrict__ dy, const __nv_bfloat16* __restrict__ a3, int rows_pad, int count,
                MlpArch A, const float* __restrict__ loss_part, float* __restrict__ grad, float* __restrict__ loss)
{
    __shared__ float sh[32];
    const int n = blockIdx.x;
    float acc = 0.f;
    if (n < A.h3) {
        for (int b = threadIdx.x; b < rows_pad; b += blockDim.x)
            acc = fmaf(dy[b], __bfloat162float(a3[static_cast<size_t>(b) * A.h3 + n]), acc);
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) grad[A.ow4 + n] = acc;
    } else if (n == A.h3) {
        for (int b = threadIdx.x; b < rows_pad; b += blockDim.x) acc += dy[b];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) grad[A.ob4] = acc;
    } else {
        for (int b = threadIdx.x; b < rows_pad; b += blockDim.x) acc += loss_part[b];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) *loss = acc / static_cast<float>(count);
    }
}

// Adam (Kingma & Ba, 2015) with bias correction, step t >= 1.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, int t)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, static_cast<float>(t)));
    const float vh = vi / (1.f - powf(b2, static_cast<float>(t)));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
}

// Minibatch gather: theta rows and targets of idx[b0 .. b0 + B).
__global__ void k_mlp_gather(const float* __restrict__ theta, const float* __restrict__ target,
                             const int* __restrict__ idx, int b0, int B, int dof,
                             float* __restrict__ th_out, float* __restrict__ t_out)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int s = idx[b0 + b];
    for (int j = 0; j < dof; ++j) th_out[static_cast<size_t>(b) * dof + j] = theta[static_cast<size_t>(s) * dof + j];
    t_out[b] = target[s];
}

// Exact label: minimum signed distance over the self pairs (Eq. 13 reading,
// positive apart) of each configuration; one warp per configuration.
__global__ void __launch_bounds__(256)
k_self_distance(storm::Problem pb, const float* __restrict__ theta, int count, float* __restrict__ sd)
{
    extern __shared__ __align__(16) float4 s_c[];  // 8 warps x M centres
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int idx = blockIdx.x * 8 + warp;
    if (idx >= count) return;
    float4* cent = s_c + warp * pb.M;
    const float* th = theta + static_cast<size_t>(idx) * pb.d;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float pp[3] = {0.f, 0.f, 0.f};
    for (int f = 0; f <= pb.d; ++f) {
        if (f > 0) {
            const float* dh = pb.dhx + (f - 1) * 8;
            storm::dh_step(R, pp, dh[0], dh[1], dh[2], dh[3], th[f - 1] + dh[4]);
        }
        for (int s = pb.link_first[f] + lane; s < pb.link_first[f + 1]; s += 32) {
            const float4 q = pb.sph[s];
            cent[s] = make_float4(fmaf(R[0], q.x, fmaf(R[1], q.y, fmaf(R[2], q.z, pp[0]))),
                                  fmaf(R[3], q.x, fmaf(R[4], q.y, fmaf(R[5], q.z, pp[1]))),
                                  fmaf(R[6], q.x, fmaf(R[7], q.y, fmaf(R[8], q.z, pp[2]))), q.w);
        }
    }
    __syncwarp();
    float best = INFINITY;
    for (int bk = 0; bk < pb.NPB; ++bk) {
        const uint4 blk = pb.pblk[bk];
        const int na = blk.y - blk.x, total = na * static_cast<int>(blk.w);
        for (int c = lane; c < total; c += 32) {
            const float4 ca = cent[blk.x + c / blk.w], cb = cent[blk.z + c % blk.w];
            const float ex = ca.x - cb.x, ey = ca.y - cb.y, ez = ca.z - cb.z;
            best = fminf(best, sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez))) - ca.w - cb.w);
        }
    }
    for (int k = lane; k < pb.P; k += 32) {
        const uint32_t pr = pb.pairs[k];
        const float4 ca = cent[pr & 0xffff], cb = cent[pr >> 16];
        const float ex = ca.x - cb.x, ey = ca.y - cb.y, ez = ca.z - cb.z;
        best = fminf(best, sqrtf(fmaf(ex, ex, fmaf(ey, ey, ez * ez))) - ca.w - cb.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) sd[idx] = best;
}
