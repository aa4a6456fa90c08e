// Legendre contractions on the 5th-generation tensor cores (tcgen05) with
// split-BF16 operands and FP32 accumulation in tensor memory.
//
// Every operand x is carried as npieces BF16 values x = x_0 + x_1 (+ x_2),
// each the rounded residual of the previous (a 2- or 3-term split).  The
// product a b is accumulated as the sum of the piece products a_i b_j with
// i + j < npieces: 3 products (2 pieces, ~2^-16 relative) or 6 products
// (3 pieces, about FP32 accuracy).  All products of one tile accumulate into
// one FP32 tile in TMEM.
//
//   synthesis  X[j][col] = sum_q Pbar(m, p, q)[j] C[q][col]       (A = Pbar^T, B = C)
//   analysis   Y[q][col] = sum_j Pbar(m, p, q)[j] W[j][col]       (A = Pbar,   B = W)
// for each group (m, p) of rows n' = m + p + 2q (the even/odd split of the
// transforms).  The static operand (Pbar) comes pre-split and pre-arranged in
// the canonical no-swizzle K-major shared-memory layout and is fetched with
// one bulk asynchronous copy (TMA) per piece and chunk; the dynamic operand
// is split by the threads while they fill shared memory.  One thread issues
// the MMAs; a tcgen05.commit arrives on an mbarrier the block waits on.
// Every wait is bounded: on expiry the block records an error flag, waits
// (bounded) for work in flight, releases its tensor memory and stops.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "async_copy.cuh"
#include "convert.cuh"
#include "sdc_internal.h"

namespace sdc {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTileRows = 128;                       // M of every MMA

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

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared memory of one block: a control block, then npieces A chunks
// [16 rb][kbc][64] and npieces B chunks [nbc][kbc][64] (BF16).  Only the
// async proxy writes the operand areas (bulk copies), so rows of A beyond a
// partial tile hold stale finite data: they only feed accumulator rows the
// epilogue never reads.  K padding is zero in both operands' global copies.
struct TcSmem {
    uint64_t mbar_ld[2];
    uint64_t mbar_mma;
    uint32_t tmem;
    int abort;
};
constexpr int kAElems = 16 * kTcChunkKB * 64;
constexpr size_t kCtrlBytes = 128;

__host__ __device__ inline int b_elems(int nbc) { return nbc * kTcChunkKB * 64; }

// two operand stages of NP pieces each
__host__ __device__ inline size_t tc_stage_elems(int np, int nbc) {
    return static_cast<size_t>(np) * (kAElems + b_elems(nbc));
}
size_t tc_smem_bytes(int np, int nbc) { return kCtrlBytes + 2 * tc_stage_elems(np, nbc) * sizeof(__nv_bfloat16); }

// The MMAs of one chunk: kbc k-blocks, K step 16 (two core matrices).
template <int NP>
__device__ __forceinline__ void issue_chunk(const __nv_bfloat16 *abase, const __nv_bfloat16 *bbase, int belems,
                                            uint32_t tmem, int kbc, int N, bool first) {
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
                mma_bf16(tmem, ad, bd, idesc, (first && ks == 0 && prod == 0) ? 0u : 1u);
            }
    }
}

// Operands of one tile: A chunks (a_rb row blocks, chunks of a_rb * kbc core
// matrices back to back from a_src, pieces a_piece apart) and B chunks (the
// first nbc col blocks of chunks of b_cb col blocks from b_src, pieces
// b_piece apart), kb_total k blocks in chunks of kTcChunkKB.
struct TileOperands {
    const uint16_t *a_src;
    long long a_piece;
    int a_rb;
    const uint16_t *b_src;
    long long b_piece;
    int b_cb, nbc, N, kb_total;
};

// Thread 0: bulk-copy chunk c into operand stage st (mbar_ld[st]).
template <int NP>
__device__ void copy_chunk(TcSmem &sm, __nv_bfloat16 *stage0, size_t stage_elems, int belems, const TileOperands &o,
                           int c, int st) {
    const int c0 = c * kTcChunkKB, kbc = min(kTcChunkKB, o.kb_total - c0);
    __nv_bfloat16 *sa = stage0 + st * stage_elems, *sb = sa + NP * kAElems;
    const uint32_t abytes = static_cast<uint32_t>(o.a_rb) * kbc * 128;
    const uint32_t bbytes = static_cast<uint32_t>(o.nbc) * kbc * 128;
    expect_tx(&sm.mbar_ld[st], NP * (abytes + bbytes));
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        bulk_copy(sa + i * kAElems, o.a_src + i * o.a_piece + static_cast<long long>(o.a_rb) * 64 * c0, abytes,
                  &sm.mbar_ld[st]);
        bulk_copy(sb + i * belems, o.b_src + i * o.b_piece + static_cast<long long>(o.b_cb) * 64 * c0, bbytes,
                  &sm.mbar_ld[st]);
    }
}

// The chunks of one tile, two operand stages deep: chunk c + 2 is copied while
// the block finishes chunk c + 1.  Every chunk's MMAs start a fresh TMEM
// accumulator (the tensor core's own accumulation spans at most kTcChunkKB k
// blocks along K) that the block adds into acc in FP32 registers (row =
// thread, columns 8 cb + u) before the next chunk's MMAs.  Bounded waits: on
// expiry the flag gets `code`, thread 0 waits once more (bounded) for copies
// and MMAs in flight and the tile is abandoned (returns false).
template <int NP, int NBC>
__device__ bool tile_chunks(TcSmem &sm, __nv_bfloat16 *stage0, int belems, const TileOperands &o, int *err,
                            int code, float (&acc)[NBC][8]) {
    const int warp = threadIdx.x >> 5;
    const size_t stage_elems = tc_stage_elems(NP, o.nbc);
#pragma unroll
    for (int cb = 0; cb < NBC; ++cb)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[cb][u] = 0.f;
    const int nch = (o.kb_total + kTcChunkKB - 1) / kTcChunkKB;
    if (threadIdx.x == 0) {
        copy_chunk<NP>(sm, stage0, stage_elems, belems, o, 0, 0);
        if (nch > 1) copy_chunk<NP>(sm, stage0, stage_elems, belems, o, 1, 1);
    }
    for (int c = 0; c < nch; ++c) {
        const int st = c & 1;
        if (threadIdx.x == 0) {
            const bool landed = mbar_wait(&sm.mbar_ld[st], (c >> 1) & 1);
            bool done = false;
            if (landed) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const __nv_bfloat16 *sa = stage0 + st * stage_elems;
                issue_chunk<NP>(sa, sa + NP * kAElems, belems, sm.tmem,
                                min(kTcChunkKB, o.kb_total - c * kTcChunkKB), o.N, true);
                mma_commit(&sm.mbar_mma);
                done = mbar_wait(&sm.mbar_mma, c & 1);
            }
            if (done && c + 2 < nch) copy_chunk<NP>(sm, stage0, stage_elems, belems, o, c + 2, st);
            if (!done) {                        // let work in flight land (bounded) and give up the tile
                atomicExch(err, landed ? code + 1 : code);
                sm.abort = 1;
                if (landed) mbar_wait(&sm.mbar_mma, c & 1);
                else mbar_wait(&sm.mbar_ld[st], (c >> 1) & 1);
                if (c + 1 < nch) mbar_wait(&sm.mbar_ld[st ^ 1], ((c + 1) >> 1) & 1);
            }
        }
        __syncthreads();
        if (sm.abort) return false;
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int cb = 0; cb < NBC; ++cb) {
            if (cb < o.nbc) {
                float v[8];
                tmem_ld8(sm.tmem + (static_cast<uint32_t>(warp * 32) << 16) + cb * 8, v);
#pragma unroll
                for (int u = 0; u < 8; ++u) acc[cb][u] += v[u];
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();                        // TMEM read before the next chunk overwrites it
    }
    return true;
}

__device__ __forceinline__ void tc_prologue(TcSmem &sm, uint32_t ncols) {
    if (threadIdx.x == 0) {
        mbar_init(&sm.mbar_ld[0], 1);
        mbar_init(&sm.mbar_ld[1], 1);
        mbar_init(&sm.mbar_mma, 1);
        mbar_init_fence();
        sm.abort = 0;
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

__device__ __forceinline__ void tc_epilogue_free(TcSmem &sm, uint32_t ncols) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// Analysis projection: one block per tile (m, p, rows q0..q0+nrows), all B
// states.  Columns col = b*10 + g*2 + (re, im) of W = F2[b][m][j][g][p],
// pre-split by k2_split_w_staged or k2_split_w.  Output Y[b][e][g] (float2),
// e = ext_offset(m) + p + 2q.
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(kTcThreads) k3_tc(TcTables tc, Dims d, int B, float2 *__restrict__ y) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    const TcTile3 t = tc.tiles3[blockIdx.x];
    const int ncols = 10 * B;
    const int N = (ncols + 15) / 16 * 16;
    const int nbc = N / 8;                      // column blocks
    const int belems = b_elems(nbc);
    __nv_bfloat16 *stage0 = reinterpret_cast<__nv_bfloat16 *>(smem_raw + kCtrlBytes);
    const uint32_t tcols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
    const int T = d.T;
    const int kjb = tc.kj / 8;
    tc_prologue(sm, tcols);
    const long long gbase = static_cast<long long>(2 * t.m + t.p) * kNbc3 * kjb * 64;
    const TileOperands o{tc.a3 + t.aoff, tc.elems3, t.nrb, tc.wb + gbase, tc.wb_elems, kNbc3, nbc, N, kjb};
    float acc[kNbc3][8];
    if (tile_chunks<NP, kNbc3>(sm, stage0, belems, o, tc.err, 1, acc)) {
        const int r = threadIdx.x;
        const int q = t.q0 + r;
        const int e = ext_offset(T, t.m) + t.p + 2 * q;
        if (r < t.nrows) {
#pragma unroll
            for (int cb = 0; cb < kNbc3; ++cb)
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const int c = cb * 8 + u;
                    if (cb < nbc && c < ncols) {
                        const int b = c / 10, g = (c - b * 10) / 2;
                        y[(static_cast<size_t>(b) * d.next + e) * 5 + g] = make_float2(acc[cb][u], acc[cb][u + 1]);
                    }
                }
        }
    }
    tc_epilogue_free(sm, tcols);
}

// ---------------------------------------------------------------------------
// Synthesis: one block per tile (m, p, latitudes j0..j0+nj), all B states.
// Columns col = b*8 + f*2 + (re, im) of the prepared coefficients C[q][col]
// (fields zeta, Phi', U, V as in the FP64/FP32 synthesis), pre-split by
// k1_prep_split.  Output F1[b][j][m][p][f] (float2).
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(kTcThreads) k1_tc(TcTables tc, Dims d, int B, float2 *__restrict__ f1) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    const TcTile1 t = tc.tiles1[blockIdx.x];
    const int ncols = 8 * B;
    const int N = (ncols + 15) / 16 * 16;
    const int nbc = N / 8;
    const int belems = b_elems(nbc);
    __nv_bfloat16 *stage0 = reinterpret_cast<__nv_bfloat16 *>(smem_raw + kCtrlBytes);
    const uint32_t tcols = N <= 32 ? 32u : 64u;
    const int T = d.T;
    const int m = t.m;
    tc_prologue(sm, tcols);
    const TileOperands o{tc.a1 + t.aoff, tc.elems1, t.njb, tc.cb + tc.cb_off[2 * m + t.p], tc.cb_elems, kNbc1, nbc, N,
                         t.KR / 8};
    float acc[kNbc1][8];
    if (tile_chunks<NP, kNbc1>(sm, stage0, belems, o, tc.err, 3, acc)) {
        const int r = threadIdx.x;
        const int j = t.j0 + r;
        if (r < t.nj) {
#pragma unroll
            for (int cb = 0; cb < kNbc1; ++cb) {
                if (cb < B) {
                    float4 *o = reinterpret_cast<float4 *>(f1 + (static_cast<size_t>(cb) * d.J2 + j) * 8 * (T + 1) +
                                                           (2 * m + t.p) * 4);
                    o[0] = make_float4(acc[cb][0], acc[cb][1], acc[cb][2], acc[cb][3]);
                    o[1] = make_float4(acc[cb][4], acc[cb][5], acc[cb][6], acc[cb][7]);
                }
            }
        }
    }
    tc_epilogue_free(sm, tcols);
}

// W^T pieces of the projection, one thread per (group, col block, k block):
// 8 columns x 8 latitudes of F2 (zero beyond B states and J2 latitudes),
// split and written as NP core matrices.  Reads the FP32 F2 layout
// [b][m][j][g][parity] straight from global memory (used where the staged
// variant below does not fit its shared memory).
template <int NP>
__global__ void k2_split_w(TcTables tc, Dims d, int B, int nbc, const float2 *__restrict__ f2) {
    const int kjb = tc.kj / 8;
    const int per_group = nbc * kjb;
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= 2LL * (d.T + 1) * per_group) return;
    const int g = static_cast<int>(idx / per_group);
    const int rem = static_cast<int>(idx - static_cast<long long>(g) * per_group);
    const int cb = rem / kjb, kb = rem - cb * kjb;
    const int m = g >> 1, p = g & 1;
    const int T = d.T, J2 = d.J2;
    const int c0 = kb / kTcChunkKB * kTcChunkKB, kbc = min(kTcChunkKB, kjb - c0);
    // all 32 loads first (clamped to valid addresses), then the zeros of
    // missing states and latitudes: nothing waits between the loads
    float2 w[4][8];
    bool live[4];
#pragma unroll
    for (int cp = 0; cp < 4; ++cp) {
        const int c = cb * 8 + 2 * cp;          // even: (re, im) of one (b, g) pair
        const int b = c / 10;
        live[cp] = b < B;
        const int bb = live[cp] ? b : 0, gg = live[cp] ? (c - 10 * b) / 2 : 0;
        // F2[b][m][j][g][parity]: latitude stride of ten values
        const float2 *src = f2 + (static_cast<size_t>(bb) * (T + 1) + m) * J2 * 10 + gg * 2 + p;
#pragma unroll
        for (int kr = 0; kr < 8; ++kr) w[cp][kr] = src[static_cast<size_t>(min(kb * 8 + kr, J2 - 1)) * 10];
    }
    float v[8][8];                              // [column in block][latitude in k block]
#pragma unroll
    for (int cp = 0; cp < 4; ++cp)
#pragma unroll
        for (int kr = 0; kr < 8; ++kr) {
            const bool ok = live[cp] && kb * 8 + kr < J2;
            v[2 * cp][kr] = ok ? w[cp][kr].x : 0.f;
            v[2 * cp + 1][kr] = ok ? w[cp][kr].y : 0.f;
        }
    uint16_t *dst = tc.wb + static_cast<long long>(g) * kNbc3 * kjb * 64 + static_cast<long long>(c0) * kNbc3 * 64 +
                    (cb * kbc + kb - c0) * 64;
#pragma unroll
    for (int cr = 0; cr < 8; ++cr) {
        uint4 out[NP];
        split8<NP>(v[cr], out);
#pragma unroll
        for (int i = 0; i < NP; ++i) *reinterpret_cast<uint4 *>(dst + i * tc.wb_elems + cr * 8) = out[i];
    }
}

// The same split with one block per order m: the ring's output of this order
// for every state (F2[b][m][j][g][parity], contiguous per state) is staged in
// shared memory with 16-byte copies, then a thread builds the 8 columns x 8
// latitudes of one (parity, column block, k block) item from there.  Items
// run parity-fastest, then column block, so the lanes of a warp read
// neighbouring values of the same latitude records instead of records eight
// latitudes apart.  Used while the B states' records fit kSplitStageMax.
constexpr size_t kSplitStageMax = 100 * 1024;   // two blocks per SM (T511 with four states measured slower staged)

template <int NP>
__global__ void __launch_bounds__(256) k2_split_w_staged(TcTables tc, Dims d, int B, int nbc,
                                                         const float2 *__restrict__ f2) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *wm = reinterpret_cast<float2 *>(smem_raw);   // [B][J2][10]
    const int m = blockIdx.x;
    const int T = d.T, J2 = d.J2;
    const int kjb = tc.kj / 8;
    for (int b = 0; b < B; ++b) {                        // 10 J2 float2 = 5 J2 16-byte pieces per state
        const float4 *src = reinterpret_cast<const float4 *>(f2 + (static_cast<size_t>(b) * (T + 1) + m) * J2 * 10);
        float4 *dst = reinterpret_cast<float4 *>(wm + static_cast<size_t>(b) * J2 * 10);
        for (int i = threadIdx.x; i < 5 * J2; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int items = 2 * nbc * kjb;
    for (int it = threadIdx.x; it < items; it += blockDim.x) {
        const int p = it & 1, rest = it >> 1;
        const int cb = rest % nbc, kb = rest / nbc;
        float v[8][8];                                   // [column in block][latitude in k block]
#pragma unroll
        for (int cp = 0; cp < 4; ++cp) {
            const int c = cb * 8 + 2 * cp;               // even: (re, im) of one (b, g) pair
            const int b = c / 10, gg = (c - 10 * b) / 2;
#pragma unroll
            for (int kr = 0; kr < 8; ++kr) {
                const int lat = kb * 8 + kr;
                float2 w = make_float2(0.f, 0.f);
                if (b < B && lat < J2) w = wm[(static_cast<size_t>(b) * J2 + lat) * 10 + gg * 2 + p];
                v[2 * cp][kr] = w.x;
                v[2 * cp + 1][kr] = w.y;
            }
        }
        const int g = 2 * m + p;
        const int c0 = kb / kTcChunkKB * kTcChunkKB, kbc = min(kTcChunkKB, kjb - c0);
        uint16_t *dst = tc.wb + static_cast<long long>(g) * kNbc3 * kjb * 64 + static_cast<long long>(c0) * kNbc3 * 64 +
                        (cb * kbc + kb - c0) * 64;
#pragma unroll
        for (int cr = 0; cr < 8; ++cr) {
            uint4 out[NP];
            split8<NP>(v[cr], out);
#pragma unroll
            for (int i = 0; i < NP; ++i) *reinterpret_cast<uint4 *>(dst + i * tc.wb_elems + cr * 8) = out[i];
        }
    }
}

// Synthesis coefficients, one thread per (extended row e, state b): the
// FP32 values (zeta, Phi', U, V) of degree n' (the wind factors as in the
// FP64/FP32 synthesis), split into NP pieces at row q of column block b.
template <int NP>
__global__ void k1_prep_split(TcTables tc, const double2 *__restrict__ states, long long sstride, Dims d,
                              const double *__restrict__ syn, const int *__restrict__ row_m) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (e >= d.next) return;
    const int T = d.T, nc = d.ncoef;
    const int m = row_m[e];
    const int ne = e - ext_offset(T, m);
    const int n = m + ne;
    const int off = order_offset(T, m);
    const double2 *st = states + b * sstride;
    // loads from clamped degrees first, then zeros outside m..T: no load waits on a branch
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
    const float x[8] = {f64_to_f32_rn(z0.x),             // narrowed on the integer pipe (convert.cuh)
                        f64_to_f32_rn(z0.y),
                        f64_to_f32_rn(p0.x),
                        f64_to_f32_rn(p0.y),
                        f64_to_f32_rn(-c0 * d0.y - c1 * zm.x - c2 * zp.x),
                        f64_to_f32_rn(c0 * d0.x - c1 * zm.y - c2 * zp.y),
                        f64_to_f32_rn(-c0 * z0.y + c1 * dm.x + c2 * dp.x),
                        f64_to_f32_rn(c0 * z0.x + c1 * dm.y + c2 * dp.y)};
    const int p = ne & 1, q = ne >> 1;
    const int krb = tc_group_krows(T, m, p) / 8;
    const int kb = q >> 3, kr = q & 7;
    const int cc0 = kb / kTcChunkKB * kTcChunkKB, kbc = min(kTcChunkKB, krb - cc0);
    uint16_t *dst = tc.cb + tc.cb_off[2 * m + p] + static_cast<long long>(cc0) * kNbc1 * 64 +
                    (b * kbc + kb - cc0) * 64 + kr;
#pragma unroll
    for (int cr = 0; cr < 8; ++cr) {
        float r = x[cr];
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            const __nv_bfloat16 h = __float2bfloat16_rn(r);
            dst[i * tc.cb_elems + cr * 8] = __bfloat16_as_ushort(h);
            r -= __bfloat162float(h);
        }
    }
}

}  // namespace

cudaError_t configure_tc_kernels() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f, int bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    set(reinterpret_cast<const void *>(k3_tc<2>), (int)tc_smem_bytes(2, kNbc3));
    set(reinterpret_cast<const void *>(k3_tc<3>), (int)tc_smem_bytes(3, kNbc3));
    set(reinterpret_cast<const void *>(k1_tc<2>), (int)tc_smem_bytes(2, kNbc1));
    set(reinterpret_cast<const void *>(k1_tc<3>), (int)tc_smem_bytes(3, kNbc1));
    set(reinterpret_cast<const void *>(k2_split_w_staged<2>), (int)kSplitStageMax);
    set(reinterpret_cast<const void *>(k2_split_w_staged<3>), (int)kSplitStageMax);
    return e;
}

cudaError_t launch_tc_synthesis(const TcTables &tc, const Dims &d, int B, const double2 *states, long long sstride,
                                const double *syn, const int *row_m, float2 *f1, cudaStream_t s, int *launches) {
    if (B < 1 || B > kMaxNodes) return cudaErrorInvalidValue;
    const int nbc = (8 * B + 15) / 16 * 2;
    const dim3 gp((d.next + 127) / 128, B);
    if (tc.npieces == 2) {
        k1_prep_split<2><<<gp, 128, 0, s>>>(tc, states, sstride, d, syn, row_m);
        k1_tc<2><<<tc.ntiles1, kTcThreads, tc_smem_bytes(2, nbc), s>>>(tc, d, B, f1);
    } else {
        k1_prep_split<3><<<gp, 128, 0, s>>>(tc, states, sstride, d, syn, row_m);
        k1_tc<3><<<tc.ntiles1, kTcThreads, tc_smem_bytes(3, nbc), s>>>(tc, d, B, f1);
    }
    if (launches) *launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_tc_projection(const TcTables &tc, const Dims &d, int B, const float2 *f2, float2 *y,
                                 cudaStream_t s, int *launches) {
    if (B < 1 || B > kMaxNodes) return cudaErrorInvalidValue;
    const int nbc = (10 * B + 15) / 16 * 2;
    const long long nsplit = 2LL * (d.T + 1) * nbc * (tc.kj / 8);
    const unsigned gs = static_cast<unsigned>((nsplit + 127) / 128);
    const size_t stage = static_cast<size_t>(B) * d.J2 * 10 * sizeof(float2);
    const bool staged = stage <= kSplitStageMax;
    if (tc.npieces == 2) {
        if (staged) k2_split_w_staged<2><<<d.T + 1, 256, stage, s>>>(tc, d, B, nbc, f2);
        else k2_split_w<2><<<gs, 128, 0, s>>>(tc, d, B, nbc, f2);
        k3_tc<2><<<tc.ntiles3, kTcThreads, tc_smem_bytes(2, nbc), s>>>(tc, d, B, y);
    } else {
        if (staged) k2_split_w_staged<3><<<d.T + 1, 256, stage, s>>>(tc, d, B, nbc, f2);
        else k2_split_w<3><<<gs, 128, 0, s>>>(tc, d, B, nbc, f2);
        k3_tc<3><<<tc.ntiles3, kTcThreads, tc_smem_bytes(3, nbc), s>>>(tc, d, B, y);
    }
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace sdc
