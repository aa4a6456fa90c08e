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

#include "sdc_internal.h"

namespace sdc {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcMaxPieces = 3;
constexpr int kTileRows = 128;                       // M of every MMA
constexpr uint32_t kWaitLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

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

__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
    }
    return done != 0;
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void expect_tx(uint64_t *mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
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
    uint64_t mbar_ld;
    uint64_t mbar_mma;
    uint32_t tmem;
    int abort;
};
constexpr int kAElems = 16 * kTcChunkKB * 64;
constexpr size_t kCtrlBytes = 128;

__host__ __device__ inline int b_elems(int nbc) { return nbc * kTcChunkKB * 64; }

size_t tc_smem_bytes(int np, int nbc) {
    return kCtrlBytes + static_cast<size_t>(np) * (kAElems + b_elems(nbc)) * sizeof(__nv_bfloat16);
}

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

// Thread 0 only: for every chunk of kb_total k blocks, bulk-copy the NP
// pieces of the A chunk (a_rb row blocks, chunks of a_rb * kbc core
// matrices back to back from a_src) and of the B chunk (the first nbc col
// blocks of a chunk of b_cb col blocks from b_src), then issue its MMAs and
// wait for them before the next copy overwrites the operands.  Returns false
// (flag set) if a bounded wait expired; it then waits once more, bounded,
// for work still in flight.
template <int NP>
__device__ bool run_chunks(TcSmem &sm, __nv_bfloat16 *sa, __nv_bfloat16 *sb, int belems, const uint16_t *a_src,
                           long long a_piece, int a_rb, const uint16_t *b_src, long long b_piece, int b_cb, int nbc,
                           int N, int kb_total, int *err, int code) {
    int chunk = 0;
    for (int c0 = 0; c0 < kb_total; c0 += kTcChunkKB, ++chunk) {
        const int kbc = min(kTcChunkKB, kb_total - c0);
        const uint32_t abytes = static_cast<uint32_t>(a_rb) * kbc * 128;
        const uint32_t bbytes = static_cast<uint32_t>(nbc) * kbc * 128;
        expect_tx(&sm.mbar_ld, NP * (abytes + bbytes));
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            bulk_copy(sa + i * kAElems, a_src + i * a_piece + static_cast<long long>(a_rb) * 64 * c0, abytes,
                      &sm.mbar_ld);
            bulk_copy(sb + i * belems, b_src + i * b_piece + static_cast<long long>(b_cb) * 64 * c0, bbytes,
                      &sm.mbar_ld);
        }
        if (!mbar_wait(&sm.mbar_ld, chunk & 1)) {
            atomicExch(err, code);
            mbar_wait(&sm.mbar_ld, chunk & 1);
            return false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        issue_chunk<NP>(sa, sb, belems, sm.tmem, kbc, N, chunk == 0);
        mma_commit(&sm.mbar_mma);
        if (!mbar_wait(&sm.mbar_mma, chunk & 1)) {
            atomicExch(err, code + 1);
            mbar_wait(&sm.mbar_mma, chunk & 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tc_prologue(TcSmem &sm, uint32_t ncols) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar_ld)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar_mma)));
        asm volatile("fence.mbarrier_init.release.cluster;");
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
// states.  Columns col = b*10 + g*2 + (re, im) of W = F2[b][m][g][p][j],
// pre-split by k2_split_w.  Output Y[b][e][g] (float2), e = ext_offset(m) + p + 2q.
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
    __nv_bfloat16 *sa = reinterpret_cast<__nv_bfloat16 *>(smem_raw + kCtrlBytes);
    __nv_bfloat16 *sb = sa + NP * kAElems;
    const uint32_t tcols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
    const int T = d.T;
    const int kjb = tc.kj / 8;
    tc_prologue(sm, tcols);
    if (threadIdx.x == 0) {
        const long long gbase = static_cast<long long>(2 * t.m + t.p) * kNbc3 * kjb * 64;
        if (!run_chunks<NP>(sm, sa, sb, belems, tc.a3 + t.aoff, tc.elems3, t.nrb, tc.wb + gbase, tc.wb_elems,
                            kNbc3, nbc, N, kjb, tc.err, 1))
            sm.abort = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!sm.abort) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int r = warp * 32 + lane;
        const int q = t.q0 + r;
        const int e = ext_offset(T, t.m) + t.p + 2 * q;
        float v[8];
        for (int cb = 0; cb < nbc; ++cb) {
            tmem_ld8(sm.tmem + (static_cast<uint32_t>(warp * 32) << 16) + cb * 8, v);
            if (r < t.nrows) {
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    const int c = cb * 8 + u;
                    if (c < ncols) {
                        const int b = c / 10, g = (c - b * 10) / 2;
                        y[(static_cast<size_t>(b) * d.next + e) * 5 + g] = make_float2(v[u], v[u + 1]);
                    }
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
// k1_prep_split.  Output F1[b][j][f][p][m] (float2).
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
    __nv_bfloat16 *sa = reinterpret_cast<__nv_bfloat16 *>(smem_raw + kCtrlBytes);
    __nv_bfloat16 *sb = sa + NP * kAElems;
    const uint32_t tcols = N <= 32 ? 32u : 64u;
    const int T = d.T;
    const int m = t.m;
    tc_prologue(sm, tcols);
    if (threadIdx.x == 0) {
        if (!run_chunks<NP>(sm, sa, sb, belems, tc.a1 + t.aoff, tc.elems1, t.njb, tc.cb + tc.cb_off[2 * m + t.p],
                            tc.cb_elems, kNbc1, nbc, N, t.KR / 8, tc.err, 3))
            sm.abort = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (!sm.abort) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int r = warp * 32 + lane;
        const int j = t.j0 + r;
        float v[8];
        for (int cb = 0; cb < nbc; ++cb) {
            tmem_ld8(sm.tmem + (static_cast<uint32_t>(warp * 32) << 16) + cb * 8, v);
            if (r < t.nj && cb < B) {
                float2 *o = f1 + (static_cast<size_t>(cb) * d.J2 + j) * 8 * (T + 1) + t.p * (T + 1) + m;
#pragma unroll
                for (int f = 0; f < 4; ++f) o[f * 2 * (T + 1)] = make_float2(v[2 * f], v[2 * f + 1]);
            }
        }
    }
    tc_epilogue_free(sm, tcols);
}

// W^T pieces of the projection, one thread per (group, col block, k block):
// 8 columns x 8 latitudes of F2 (zero beyond B states and J2 latitudes),
// split and written as NP core matrices.
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
    float v[8][8];                              // [column in block][latitude in k block]
#pragma unroll
    for (int cp = 0; cp < 4; ++cp) {
        const int c = cb * 8 + 2 * cp;          // even: (re, im) of one (b, g) pair
        const int b = c / 10;
        const float2 *src = nullptr;
        if (b < B) src = f2 + ((static_cast<size_t>(b) * (T + 1) + m) * 5 + (c - 10 * b) / 2) * 2 * J2 + p * J2;
#pragma unroll
        for (int kr = 0; kr < 8; ++kr) {
            const int j = kb * 8 + kr;
            const float2 w = (src && j < J2) ? src[j] : make_float2(0.f, 0.f);
            v[2 * cp][kr] = w.x;
            v[2 * cp + 1][kr] = w.y;
        }
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
    auto ld = [&](int f, int k) -> double2 {
        return (k >= m && k <= T) ? st[f * nc + off + k - m] : make_double2(0.0, 0.0);
    };
    const double2 z0 = ld(F_ZETA, n), zm = ld(F_ZETA, n - 1), zp = ld(F_ZETA, n + 1);
    const double2 d0 = ld(F_DIV, n), dm = ld(F_DIV, n - 1), dp = ld(F_DIV, n + 1);
    const double2 p0 = ld(F_PHI, n);
    const double c0 = syn[3 * e], c1 = syn[3 * e + 1], c2 = syn[3 * e + 2];
    const float x[8] = {float(z0.x),
                        float(z0.y),
                        float(p0.x),
                        float(p0.y),
                        float(-c0 * d0.y - c1 * zm.x - c2 * zp.x),
                        float(c0 * d0.x - c1 * zm.y - c2 * zp.y),
                        float(-c0 * z0.y + c1 * dm.x + c2 * dp.x),
                        float(c0 * z0.x + c1 * dm.y + c2 * dp.y)};
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
    if (tc.npieces == 2) {
        k2_split_w<2><<<gs, 128, 0, s>>>(tc, d, B, nbc, f2);
        k3_tc<2><<<tc.ntiles3, kTcThreads, tc_smem_bytes(2, nbc), s>>>(tc, d, B, y);
    } else {
        k2_split_w<3><<<gs, 128, 0, s>>>(tc, d, B, nbc, f2);
        k3_tc<3><<<tc.ntiles3, kTcThreads, tc_smem_bytes(3, nbc), s>>>(tc, d, B, y);
    }
    if (launches) *launches += 2;
    return cudaGetLastError();
}

}  // namespace sdc
