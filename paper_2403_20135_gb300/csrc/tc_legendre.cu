// Legendre contractions on the 5th-generation tensor cores (tcgen05) with
// split-BF16 operands and FP32 accumulation in tensor memory.
//
// Every operand x is carried as npieces BF16 values x = x_0 + x_1 (+ x_2),
// each the rounded residual of the previous (a 2- or 3-term split).  The
// product a b is accumulated as the sum of the piece products a_i b_j with
// i + j < npieces: 3 products (2 pieces, ~2^-16 relative) or 6 products
// (3 pieces, about FP32 accuracy).
//
//   synthesis  X[j][col] = sum_q Pbar(m, p, q)[j] C[q][col]       (A = Pbar^T, B = C)
//   analysis   Y[q][col] = sum_j Pbar(m, p, q)[j] W[j][col]       (A = Pbar,   B = W)
// for each group (m, p) of rows n' = m + p + 2q (the even/odd split of the
// transforms).  The static operand (Pbar) comes pre-split and pre-arranged in
// the canonical no-swizzle K-major shared-memory layout, one contiguous bulk
// copy (TMA) per piece and K chunk.  The dynamic operand is split inside the
// kernel: the projection's W streams chunk by chunk from the ring's FP32
// output (cp.async, several chunks ahead) and is split into pieces in shared
// memory; the synthesis operand C (the coefficient combinations of the FP64
// states) is formed and split for the whole group at the start of the tile.
//
// Warp roles (192 threads): warps 0-3 split the dynamic operand and read the
// accumulators (TMEM lane = thread); one thread of warp 4 issues the bulk
// copies of the Legendre pieces into a ring of operand stages; one thread of
// warp 5 issues the MMAs.  Each K chunk (32) starts a fresh FP32 accumulator
// in TMEM (the tensor core's own accumulation spans one chunk) and warps 0-3
// add it into registers; two accumulator buffers alternate so that the MMAs
// of chunk c + 1 run while chunk c is read.  mbarriers connect the roles:
//   afull[s]  Legendre pieces of stage s landed (transaction bytes)
//   pfull[s]  dynamic pieces of stage s written (128 arrivals)
//   empty[s]  MMAs reading stage s completed (tcgen05.commit)
//   mdone[a]  accumulator buffer a complete (tcgen05.commit)
//   tfree[a]  accumulator buffer a read (128 arrivals)
// Every wait is bounded (polls and one second of the global timer) and also
// stops when another role has given up; the block then records an error flag,
// lets the copies and MMAs it issued land (bounded), frees its tensor memory
// and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "async_copy.cuh"
#include "convert.cuh"
#include "sdc_internal.h"

namespace sdc {

namespace {

constexpr int kTileRows = 128;                       // M of every MMA
constexpr int kTcWarps = 6;
constexpr int kTcThreads = 32 * kTcWarps;
constexpr int kWork = 128;                           // threads of warps 0-3
constexpr int kMaxStages = 4;
constexpr int kRawSlots = 3;                         // W chunks in flight ahead of the split
constexpr int kChunkK = 8 * kTcChunkKB;              // 32

// Shared-memory matrix descriptor (tcgen05), no swizzle: start address,
// leading byte offset = distance of core matrices along K, stride byte offset
// = distance of core matrices along M/N, descriptor version 1 (bit 46).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return static_cast<uint64_t>((saddr & 0x3FFFF) >> 4) | (static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16) |
           (static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32) | (static_cast<uint64_t>(1) << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__device__ __forceinline__ uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}

// Shared-memory writes of the generic proxy (plain stores) made visible to
// the async proxy that the tensor core reads operands through.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Named barrier over warps 0-3 with an OR reduction: every thread gets the
// same answer, so the four warps leave their loop together.
__device__ __forceinline__ bool work_sync_or(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "barrier.cta.red.or.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(v ? 1u : 0u)
        : "memory");
    return r != 0;
}

// Bounded wait that also gives up as soon as another role has set *abort.
__device__ __forceinline__ bool wait_or_abort(uint64_t *mbar, uint32_t phase, const volatile int *abort) {
    uint32_t done = 0;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
        if (!done && (it & 63u) == 63u) {
            if (*abort) break;
            if (global_ns() - t0 > kWaitNs) break;
        }
    }
    return done != 0;
}

// x = h_0 + h_1 (+ h_2): each piece the BF16 rounding of the remaining FP32
// residual (the residual of a BF16 rounding is exact in FP32).  split8 does
// this for 8 values and packs piece i of all 8 into one 16-byte word.
template <int NP>
__device__ __forceinline__ void split8(const float (&x)[8], uint4 (&out)[NP]) {
    float r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = x[k];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __nv_bfloat16 lo = __float2bfloat16_rn(r[2 * h]), hi = __float2bfloat16_rn(r[2 * h + 1]);
            r[2 * h] -= __bfloat162float(lo);
            r[2 * h + 1] -= __bfloat162float(hi);
            w[h] = static_cast<uint32_t>(__bfloat16_as_ushort(lo)) |
                   (static_cast<uint32_t>(__bfloat16_as_ushort(hi)) << 16);
        }
        out[i] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Pipeline state of one block (start of shared memory).
struct TcPipe {
    uint64_t afull[kMaxStages];
    uint64_t pfull[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t mdone[2];
    uint64_t tfree[2];
    uint64_t cready;                  // synthesis: the whole group's C pieces written
    uint32_t tmem;
    int abort;
};
constexpr size_t kCtrlBytes = 256;
static_assert(sizeof(TcPipe) <= kCtrlBytes, "pipeline state fits the control block");

constexpr int kAElems = 16 * kTcChunkKB * 64;      // one piece of one A chunk (128 rows x 32 k)

__host__ __device__ inline int b_elems(int nbc) { return nbc * kTcChunkKB * 64; }

__device__ __forceinline__ void pipe_init(TcPipe &sm, int nstages) {
    for (int s = 0; s < nstages; ++s) {
        mbar_init(&sm.afull[s], 1);
        mbar_init(&sm.pfull[s], kWork);
        mbar_init(&sm.empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
        mbar_init(&sm.mdone[a], 1);
        mbar_init(&sm.tfree[a], kWork);
    }
    mbar_init(&sm.cready, kWork);
    mbar_init_fence();
    sm.abort = 0;
}

__device__ __forceinline__ void give_up(TcPipe &sm, int *err, int code) {
    atomicCAS(err, 0, code);                          // the first cause is kept
    *reinterpret_cast<volatile int *>(&sm.abort) = 1;
}

// The MMAs of one chunk into accumulator columns tmem: kbc k-blocks, K step
// 16 (two core matrices), every piece product i + j < NP.
template <int NP>
__device__ __forceinline__ void issue_chunk(const __nv_bfloat16 *abase, const __nv_bfloat16 *bbase, int belems,
                                            uint32_t tmem, int kbc, int N) {
    const uint32_t idesc = mma_idesc(kTileRows, N);
    const uint32_t sbo = static_cast<uint32_t>(kbc) * 128;
    const uint32_t a0 = smem_u32(abase), b0 = smem_u32(bbase);
    for (int ks = 0; ks < kbc / 2; ++ks) {
        int prod = 0;
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
            for (int j = 0; i + j < NP; ++j, ++prod) {
                const uint64_t ad = smem_desc(a0 + i * kAElems * 2 + ks * 256, 128, sbo);
                const uint64_t bd = smem_desc(b0 + j * belems * 2 + ks * 256, 128, sbo);
                mma_bf16(tmem, ad, bd, idesc, (ks == 0 && prod == 0) ? 0u : 1u);
            }
    }
}

// Read the chunk's accumulator (row = thread of warps 0-3, nbc blocks of 8
// columns from column col0) and add it into acc.
template <int NBC>
__device__ __forceinline__ void tmem_accumulate(uint32_t taddr, int nbc, float (&acc)[NBC][8]) {
#pragma unroll
    for (int c0 = 0; c0 < NBC; c0 += 2) {         // two column blocks per wait keeps the registers low
        if (c0 < nbc) {
            uint32_t r[2][8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (c0 + h < NBC && c0 + h < nbc) {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[h][0]), "=r"(r[h][1]), "=r"(r[h][2]), "=r"(r[h][3]), "=r"(r[h][4]),
                                   "=r"(r[h][5]), "=r"(r[h][6]), "=r"(r[h][7])
                                 : "r"(taddr + (c0 + h) * 8));
                }
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (c0 + h < NBC && c0 + h < nbc)
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc[c0 + h][u] += __uint_as_float(r[h][u]);
        }
    }
}

__device__ __forceinline__ void tmem_alloc(TcPipe &sm, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(TcPipe &sm, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(ncols));
}

__host__ __device__ inline uint32_t tmem_cols(int N) {
    const int need = 2 * N;
    return need <= 32 ? 32u : need <= 64 ? 64u : need <= 128 ? 128u : 256u;
}

// ---- the two single-thread roles -------------------------------------------
// Warp 4, lane 0: bulk copies of the Legendre pieces of chunk c into stage
// c % S once the MMAs of chunk c - S have released it.  a_src: chunk 0 of
// piece 0; chunk c starts a_rb * 64 * kTcChunkKB * c elements further (a
// full chunk), pieces a_piece apart.
template <int NP>
__device__ void tc_producer(TcPipe &sm, __nv_bfloat16 *astage, int nstages, const uint16_t *a_src,
                            long long a_piece, int a_rb, int kb_total, int *err, int code) {
    const volatile int *abort = &sm.abort;
    const int nch = (kb_total + kTcChunkKB - 1) / kTcChunkKB;
    int c = 0;
    for (; c < nch; ++c) {
        const int s = c % nstages;
        if (c >= nstages && !wait_or_abort(&sm.empty[s], ((c / nstages) - 1) & 1, abort)) {
            if (!*abort) give_up(sm, err, code);
            break;
        }
        const int c0 = c * kTcChunkKB, kbc = min(kTcChunkKB, kb_total - c0);
        const uint32_t bytes = static_cast<uint32_t>(a_rb) * kbc * 128;
        __nv_bfloat16 *dst = astage + static_cast<size_t>(s) * NP * kAElems;
        expect_tx(&sm.afull[s], NP * bytes);
#pragma unroll
        for (int i = 0; i < NP; ++i)
            bulk_copy(dst + i * kAElems, a_src + i * a_piece + static_cast<long long>(a_rb) * 64 * c0, bytes,
                      &sm.afull[s]);
    }
    // let every issued copy land before the block can leave (bounded)
    for (int k = max(0, c - nstages); k < c; ++k) mbar_wait(&sm.afull[k % nstages], (k / nstages) & 1);
}

// Warp 5, lane 0: the MMAs of chunk c once its Legendre pieces (afull), its
// dynamic pieces (pfull, or cready once for the synthesis) and its
// accumulator buffer (tfree) are ready; commits release the stage and
// complete the buffer.
template <int NP>
__device__ void tc_issuer(TcPipe &sm, const __nv_bfloat16 *astage, const __nv_bfloat16 *bstage,
                          size_t bstage_elems, int belems, int nstages, int kb_total, int N, bool whole_b,
                          int *err, int code) {
    const volatile int *abort = &sm.abort;
    const int nch = (kb_total + kTcChunkKB - 1) / kTcChunkKB;
    int c = 0;
    bool ok = true;
    if (whole_b && !wait_or_abort(&sm.cready, 0, abort)) ok = false;
    for (; ok && c < nch; ++c) {
        const int s = c % nstages, a = c & 1;
        if (!wait_or_abort(&sm.afull[s], (c / nstages) & 1, abort) ||
            (!whole_b && !wait_or_abort(&sm.pfull[s], (c / nstages) & 1, abort)) ||
            (c >= 2 && !wait_or_abort(&sm.tfree[a], ((c >> 1) - 1) & 1, abort))) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int kbc = min(kTcChunkKB, kb_total - c * kTcChunkKB);
        const __nv_bfloat16 *b = whole_b ? bstage + static_cast<size_t>(c) * bstage_elems
                                         : bstage + static_cast<size_t>(s) * bstage_elems;
        issue_chunk<NP>(astage + static_cast<size_t>(s) * NP * kAElems, b, belems, sm.tmem + a * N, kbc, N);
        mma_commit(&sm.empty[s]);
        mma_commit(&sm.mdone[a]);
    }
    if (!ok && !*abort) give_up(sm, err, code + 1);
    // the MMAs issued so far complete before the block can free their memory (bounded)
    if (c > 0) mbar_wait(&sm.mdone[(c - 1) & 1], ((c - 1) >> 1) & 1);
}

// Warps 0-3: wait for accumulator buffer c & 1, add it into acc, release it.
template <int NBC>
__device__ __forceinline__ bool tc_consume(TcPipe &sm, int c, int N, int nbc, float (&acc)[NBC][8]) {
    const int a = c & 1;
    const bool ok = wait_or_abort(&sm.mdone[a], (c >> 1) & 1, &sm.abort);
    if (work_sync_or(!ok)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int warp = threadIdx.x >> 5;
    tmem_accumulate<NBC>(sm.tmem + (static_cast<uint32_t>(warp * 32) << 16) + a * N, nbc, acc);
    asm volatile("tcgen05.fence::before_thread_sync;");
    mbar_arrive(&sm.tfree[a]);
    return true;
}

// ---------------------------------------------------------------------------
// Analysis projection: one block per tile (m, p, rows q0..q0+nrows), all B
// states.  B operand W[j][col], col = b*10 + g*2 + (re, im), taken from the
// ring's FP32 output F2[b][m][g][p][j] chunk by chunk (32 latitudes; cp.async
// kRawSlots chunks ahead) and split into NP pieces by warps 0-3.  Output
// Y[b][e][g] (float2), e = ext_offset(m) + p + 2q.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t tc3_smem_bytes(int np, int B, int nstages) {
    const int nbc = (10 * B + 15) / 16 * 2;
    return kCtrlBytes + static_cast<size_t>(nstages) * np * (kAElems + b_elems(nbc)) * sizeof(__nv_bfloat16) +
           static_cast<size_t>(kRawSlots) * 5 * B * kChunkK * sizeof(float2);
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 2) k3_tc(TcTables tc, Dims d, int B, const float2 *__restrict__ f2,
                                                    float2 *__restrict__ y, int nstages) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcPipe &sm = *reinterpret_cast<TcPipe *>(smem_raw);
    const TcTile3 t = tc.tiles3[blockIdx.x];
    const int ncols = 10 * B;
    const int N = (ncols + 15) / 16 * 16;
    const int nbc = N / 8;
    const int belems = b_elems(nbc);
    const int kjb = tc.kj / 8;
    const int nch = (kjb + kTcChunkKB - 1) / kTcChunkKB;
    const int T = d.T, J2 = d.J2;
    const int rows = 5 * B;
    __nv_bfloat16 *astage = reinterpret_cast<__nv_bfloat16 *>(smem_raw + kCtrlBytes);
    __nv_bfloat16 *pstage = astage + static_cast<size_t>(nstages) * NP * kAElems;
    float2 *raw = reinterpret_cast<float2 *>(pstage + static_cast<size_t>(nstages) * NP * belems);
    const uint32_t tcols = tmem_cols(N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) pipe_init(sm, nstages);
    if (warp == 0) tmem_alloc(sm, tcols);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (warp == 4) {
        if (lane == 0) tc_producer<NP>(sm, astage, nstages, tc.a3 + t.aoff, tc.elems3, t.nrb, kjb, tc.err, 1);
    } else if (warp == 5) {
        if (lane == 0)
            tc_issuer<NP>(sm, astage, pstage, static_cast<size_t>(NP) * belems, belems, nstages, kjb, N, false,
                          tc.err, 1);
    } else {
        const int tid = threadIdx.x;
        auto prefetch = [&](int c) {
            if (c < nch) {
                float2 *slot = raw + static_cast<size_t>(c % kRawSlots) * rows * kChunkK;
                const int j0 = c * kChunkK;
                for (int i = tid; i < rows * kChunkK; i += kWork) {
                    const int r = i >> 5, j = j0 + (i & 31);
                    const int b = r / 5, g = r - 5 * b;
                    if (j < J2)
                        cp_async8(slot + i, f2 + ((static_cast<size_t>(b) * (T + 1) + t.m) * 5 + g) * 2 * J2 +
                                                static_cast<size_t>(t.p) * J2 + j);
                    else
                        slot[i] = make_float2(0.f, 0.f);
                }
            }
            cp_async_commit();                         // one group per chunk, empty past the end
        };
#pragma unroll
        for (int c = 0; c < kRawSlots; ++c) prefetch(c);
        float acc[kNbc3][8];
#pragma unroll
        for (int cb = 0; cb < kNbc3; ++cb)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[cb][u] = 0.f;
        bool ok = true;
        for (int c = 0; c < nch && ok; ++c) {
            const int s = c % nstages;
            cp_async_wait<kRawSlots - 1>();            // this thread's copies of chunk c
            bool bad = false;
            if (c >= nstages) bad = !wait_or_abort(&sm.empty[s], ((c / nstages) - 1) & 1, &sm.abort);
            if (work_sync_or(bad)) {                   // also: every thread's copies of chunk c are visible
                ok = false;
                break;
            }
            const int kbc = min(kTcChunkKB, kjb - c * kTcChunkKB);
            const float2 *slot = raw + static_cast<size_t>(c % kRawSlots) * rows * kChunkK;
            __nv_bfloat16 *ps = pstage + static_cast<size_t>(s) * NP * belems;
            for (int it = tid; it < N * kbc; it += kWork) {
                const int col = it / kbc, kb = it - col * kbc;
                float v[8];
                if (col < ncols) {
                    const float4 *src = reinterpret_cast<const float4 *>(slot + (col >> 1) * kChunkK + kb * 8);
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const float4 q = src[h];
                        v[2 * h] = (col & 1) ? q.y : q.x;
                        v[2 * h + 1] = (col & 1) ? q.w : q.z;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) v[e] = 0.f;
                }
                uint4 out[NP];
                split8<NP>(v, out);
                const int cb = col >> 3, cr = col & 7;
#pragma unroll
                for (int i = 0; i < NP; ++i)
                    *reinterpret_cast<uint4 *>(ps + static_cast<size_t>(i) * belems + (cb * kbc + kb) * 64 + cr * 8) =
                        out[i];
            }
            fence_async_smem();
            mbar_arrive(&sm.pfull[s]);
            work_sync_or(false);                       // every thread is done with raw slot c: refill it
            prefetch(c + kRawSlots);
            if (c >= 1 && !tc_consume<kNbc3>(sm, c - 1, N, nbc, acc)) ok = false;
        }
        if (ok) ok = tc_consume<kNbc3>(sm, nch - 1, N, nbc, acc);
        cp_async_wait<0>();
        if (!ok) {
            if (tid == 0) give_up(sm, tc.err, 3);
        } else if (tid < t.nrows) {
            const int q = t.q0 + tid;
            const int e = ext_offset(T, t.m) + t.p + 2 * q;
#pragma unroll
            for (int cb = 0; cb < kNbc3; ++cb)
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const int col = cb * 8 + u;
                    if (cb < nbc && col < ncols) {
                        const int b = col / 10, g = (col - b * 10) / 2;
                        y[(static_cast<size_t>(b) * d.next + e) * 5 + g] = make_float2(acc[cb][u], acc[cb][u + 1]);
                    }
                }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) tmem_free(sm, tcols);
}

// ---------------------------------------------------------------------------
// Synthesis: one block per tile (m, p, latitudes j0..j0+nj), all B states.
// B operand C[q][col], col = b*8 + f*2 + (re, im): the FP32 values of zeta,
// Phi' and the wind combinations U, V of degree n' = m + p + 2q (FP64
// arithmetic on the FP64 states, narrowed on the integer pipe), formed for
// the whole group by warps 0-3 while the first Legendre chunks are copied,
// then split into NP pieces chunk by chunk.  Output F1[b][j][f][p][m].
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t tc1_smem_bytes(int np, int B, int krmax, int nstages) {
    const int N = (8 * B + 15) / 16 * 16;
    const int nchmax = (krmax / 8 + kTcChunkKB - 1) / kTcChunkKB;
    return kCtrlBytes + static_cast<size_t>(nstages) * np * kAElems * sizeof(__nv_bfloat16) +
           static_cast<size_t>(nchmax) * np * b_elems(N / 8) * sizeof(__nv_bfloat16) +
           static_cast<size_t>(krmax) * N * sizeof(float);
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 2) k1_tc(TcTables tc, Dims d, int B, const double2 *__restrict__ states,
                                                    long long sstride, const double *__restrict__ syn,
                                                    float2 *__restrict__ f1, int nstages) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcPipe &sm = *reinterpret_cast<TcPipe *>(smem_raw);
    const TcTile1 t = tc.tiles1[blockIdx.x];
    const int ncols = 8 * B;
    const int N = (ncols + 15) / 16 * 16;
    const int nbc = N / 8;
    const int belems = b_elems(nbc);
    const int krb = t.KR / 8;
    const int nch = (krb + kTcChunkKB - 1) / kTcChunkKB;
    const int T = d.T, nc = d.ncoef, m = t.m;
    __nv_bfloat16 *astage = reinterpret_cast<__nv_bfloat16 *>(smem_raw + kCtrlBytes);
    __nv_bfloat16 *cpieces = astage + static_cast<size_t>(nstages) * NP * kAElems;   // [chunk][NP][belems]
    float *cf = reinterpret_cast<float *>(cpieces + static_cast<size_t>(nch) * NP * belems);   // [KR][N]
    const uint32_t tcols = tmem_cols(N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) pipe_init(sm, nstages);
    if (warp == 0) tmem_alloc(sm, tcols);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (warp == 4) {
        if (lane == 0) tc_producer<NP>(sm, astage, nstages, tc.a1 + t.aoff, tc.elems1, t.njb, krb, tc.err, 5);
    } else if (warp == 5) {
        if (lane == 0)
            tc_issuer<NP>(sm, astage, cpieces, static_cast<size_t>(NP) * belems, belems, nstages, krb, N, true,
                          tc.err, 5);
    } else {
        const int tid = threadIdx.x;
        // pass 1: FP32 coefficient rows, cf[q][b*8 + f*2 + (re, im)]; zero beyond R rows and 8B columns
        for (int it = tid; it < t.KR * B; it += kWork) {
            const int q = it / B, b = it - q * B;
            float *o = cf + static_cast<size_t>(q) * N + 8 * b;
            if (q >= t.R) {
#pragma unroll
                for (int k = 0; k < 8; ++k) o[k] = 0.f;
                continue;
            }
            const int ne = t.p + 2 * q, n = m + ne;
            const int e = ext_offset(T, m) + ne;
            const int off = order_offset(T, m);
            const double2 *st = states + b * sstride;
            // loads from clamped degrees first, then zeros outside m..T
            auto ldc = [&](int f, int k) { return st[f * nc + off + min(max(k, m), T) - m]; };
            auto in = [&](int k) { return k >= m && k <= T; };
            double2 z0 = ldc(F_ZETA, n), zm = ldc(F_ZETA, n - 1), zp = ldc(F_ZETA, n + 1);
            double2 d0 = ldc(F_DIV, n), dm = ldc(F_DIV, n - 1), dp = ldc(F_DIV, n + 1);
            double2 p0 = ldc(F_PHI, n);
            const double c0 = syn[3 * e], c1 = syn[3 * e + 1], c2 = syn[3 * e + 2];
            const double2 zero = make_double2(0.0, 0.0);
            if (!in(n)) z0 = d0 = p0 = zero;
            if (!in(n - 1)) zm = dm = zero;
            if (!in(n + 1)) zp = dp = zero;
            o[0] = f64_to_f32_rn(z0.x);
            o[1] = f64_to_f32_rn(z0.y);
            o[2] = f64_to_f32_rn(p0.x);
            o[3] = f64_to_f32_rn(p0.y);
            o[4] = f64_to_f32_rn(-c0 * d0.y - c1 * zm.x - c2 * zp.x);
            o[5] = f64_to_f32_rn(c0 * d0.x - c1 * zm.y - c2 * zp.y);
            o[6] = f64_to_f32_rn(-c0 * z0.y + c1 * dm.x + c2 * dp.x);
            o[7] = f64_to_f32_rn(c0 * z0.x + c1 * dm.y + c2 * dp.y);
        }
        for (int it = tid; it < t.KR * (N - ncols); it += kWork) {
            const int q = it / (N - ncols), k = it - q * (N - ncols);
            cf[static_cast<size_t>(q) * N + ncols + k] = 0.f;
        }
        work_sync_or(false);
        // pass 2: 8 consecutive rows of one column -> NP 16-byte piece words
        for (int it = tid; it < N * krb; it += kWork) {
            const int col = it / krb, kbg = it - col * krb;
            const int c = kbg / kTcChunkKB, kb = kbg - c * kTcChunkKB;
            const int kbc = min(kTcChunkKB, krb - c * kTcChunkKB);
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = cf[static_cast<size_t>(kbg * 8 + e) * N + col];
            uint4 out[NP];
            split8<NP>(v, out);
            __nv_bfloat16 *dst = cpieces + static_cast<size_t>(c) * NP * belems + ((col >> 3) * kbc + kb) * 64 +
                                 (col & 7) * 8;
#pragma unroll
            for (int i = 0; i < NP; ++i) *reinterpret_cast<uint4 *>(dst + static_cast<size_t>(i) * belems) = out[i];
        }
        fence_async_smem();
        mbar_arrive(&sm.cready);
        float acc[kNbc1][8];
#pragma unroll
        for (int cb = 0; cb < kNbc1; ++cb)
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[cb][u] = 0.f;
        bool ok = true;
        for (int c = 0; c < nch && ok; ++c) ok = tc_consume<kNbc1>(sm, c, N, nbc, acc);
        if (!ok) {
            if (tid == 0) give_up(sm, tc.err, 7);
        } else if (tid < t.nj) {
            const int j = t.j0 + tid;
#pragma unroll
            for (int cb = 0; cb < kNbc1; ++cb) {
                if (cb < B) {
                    float2 *o = f1 + (static_cast<size_t>(cb) * d.J2 + j) * 8 * (T + 1) + t.p * (T + 1) + m;
#pragma unroll
                    for (int f = 0; f < 4; ++f) o[f * 2 * (T + 1)] = make_float2(acc[cb][2 * f], acc[cb][2 * f + 1]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) tmem_free(sm, tcols);
}

// Operand stages per block: the most that still lets two blocks share an SM,
// else the most that fit one block per SM.
constexpr size_t kSmemPerSm = 227 * 1024;
template <typename F>
int choose_stages(F bytes) {
    for (size_t cap : {kSmemPerSm / 2 - 1024, kSmemPerSm})
        for (int s = kMaxStages; s >= 1; --s)
            if (bytes(s) <= cap) return s;
    return 0;
}

int tc_krmax(int T) { return tc_group_krows(T, 0, 0); }

}  // namespace

cudaError_t configure_tc_kernels() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kSmemPerSm));
    };
    set(reinterpret_cast<const void *>(k3_tc<2>));
    set(reinterpret_cast<const void *>(k3_tc<3>));
    set(reinterpret_cast<const void *>(k1_tc<2>));
    set(reinterpret_cast<const void *>(k1_tc<3>));
    return e;
}

// Whether the tensor-core kernels serve B states at truncation T with np pieces.
bool tc_fits(int T, int np, int B) {
    if (B < 1 || B > kMaxNodes) return false;
    const int s3 = choose_stages([&](int s) { return tc3_smem_bytes(np, B, s); });
    const int s1 = choose_stages([&](int s) { return tc1_smem_bytes(np, B, tc_krmax(T), s); });
    return s3 >= 1 && s1 >= 1;
}

cudaError_t launch_tc_synthesis(const TcTables &tc, const Dims &d, int B, const double2 *states, long long sstride,
                                const double *syn, float2 *f1, cudaStream_t s, int *launches) {
    const int np = tc.npieces;
    const int krmax = tc_krmax(d.T);
    const int ns = choose_stages([&](int st) { return tc1_smem_bytes(np, B, krmax, st); });
    if (B < 1 || B > kMaxNodes || ns < 1) return cudaErrorInvalidValue;
    const size_t smem = tc1_smem_bytes(np, B, krmax, ns);
    if (np == 2)
        k1_tc<2><<<tc.ntiles1, kTcThreads, smem, s>>>(tc, d, B, states, sstride, syn, f1, ns);
    else
        k1_tc<3><<<tc.ntiles1, kTcThreads, smem, s>>>(tc, d, B, states, sstride, syn, f1, ns);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_tc_projection(const TcTables &tc, const Dims &d, int B, const float2 *f2, float2 *y,
                                 cudaStream_t s, int *launches) {
    const int np = tc.npieces;
    const int ns = choose_stages([&](int st) { return tc3_smem_bytes(np, B, st); });
    if (B < 1 || B > kMaxNodes || ns < 1) return cudaErrorInvalidValue;
    const size_t smem = tc3_smem_bytes(np, B, ns);
    if (np == 2)
        k3_tc<2><<<tc.ntiles3, kTcThreads, smem, s>>>(tc, d, B, f2, y, ns);
    else
        k3_tc<3><<<tc.ntiles3, kTcThreads, smem, s>>>(tc, d, B, f2, y, ns);
    if (launches) *launches += 1;
    return cudaGetLastError();
}

}  // namespace sdc
