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
// residual (the residual of a BF16 rounding is exact in FP32).  Piece i of
// element idx lives at base[i * stride + idx].
template <int NP>
__device__ __forceinline__ void split_store(float x, __nv_bfloat16 *base, int stride, int idx) {
    float r = x;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        const __nv_bfloat16 h = __float2bfloat16_rn(r);
        base[i * stride + idx] = h;
        r -= __bfloat162float(h);
    }
}

// zero [from, to) elements of a BF16 array with 16-byte stores where aligned
__device__ __forceinline__ void zero_range(__nv_bfloat16 *a, int from, int to) {
    const int vfrom = (from + 7) & ~7, vto = to & ~7;
    for (int k = from + threadIdx.x; k < min(vfrom, to); k += blockDim.x) a[k] = __float2bfloat16(0.0f);
    uint4 *v = reinterpret_cast<uint4 *>(a);
    for (int k = vfrom / 8 + threadIdx.x; k < vto / 8; k += blockDim.x) v[k] = make_uint4(0, 0, 0, 0);
    for (int k = max(vto, vfrom) + threadIdx.x; k < to; k += blockDim.x) a[k] = __float2bfloat16(0.0f);
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
// [16 rb][8 kb][64] and npieces B chunks [<= 10 rb][8 kb][64] (BF16).
struct TcSmem {
    uint64_t mbar_ld;
    uint64_t mbar_mma;
    uint32_t tmem;
    int abort;
};
constexpr int kAElems = 16 * kTcChunkKB * 64;
constexpr int kBElems = 10 * kTcChunkKB * 64;
constexpr size_t kCtrlBytes = 128;

size_t tc_smem_bytes(int np) {
    return kCtrlBytes + static_cast<size_t>(np) * (kAElems + kBElems) * sizeof(__nv_bfloat16);
}

// piece i of the A chunk at a_base + i * kAElems, of the B chunk at b_base + i * kBElems
template <int NP>
__device__ __forceinline__ __nv_bfloat16 *a_base(unsigned char *raw) {
    return reinterpret_cast<__nv_bfloat16 *>(raw + kCtrlBytes);
}
template <int NP>
__device__ __forceinline__ __nv_bfloat16 *b_base(unsigned char *raw) {
    return reinterpret_cast<__nv_bfloat16 *>(raw + kCtrlBytes) + NP * kAElems;
}

// one thread waits (bounded) on an mbarrier phase while the block sleeps at
// the barrier; returns false everywhere if the wait expired
__device__ __forceinline__ bool block_wait(TcSmem &sm, uint64_t *mbar, uint32_t phase, int *err, int code) {
    if (threadIdx.x == 0) {
        if (!mbar_wait(mbar, phase)) {
            sm.abort = 1;
            atomicExch(err, code);
            mbar_wait(mbar, phase);                 // work may still be landing: wait again (bounded)
        }
    }
    __syncthreads();
    return sm.abort == 0;
}

// The MMAs of one chunk: kbc k-blocks, K step 16 (two core matrices).
template <int NP>
__device__ __forceinline__ void issue_chunk(const __nv_bfloat16 *abase, const __nv_bfloat16 *bbase, uint32_t tmem,
                                            int kbc, int N, bool first) {
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
                const uint64_t bd = smem_desc(b0 + j * kBElems * 2 + ks * 256, 128, sbo);
                mma_bf16(tmem, ad, bd, idesc, (first && ks == 0 && prod == 0) ? 0u : 1u);
            }
    }
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
// states.  Columns col = b*10 + g*2 + (re, im) of W = F2[b][m][g][p][j].
// Output Y[b][e][g] (float2), e = ext_offset(m) + p + 2q.
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(kTcThreads) k3_tc(TcTables tc, Dims d, int B, const float2 *__restrict__ f2,
                                                    float2 *__restrict__ y) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    __nv_bfloat16 *sa = a_base<NP>(smem_raw);
    __nv_bfloat16 *sb = b_base<NP>(smem_raw);
    const TcTile3 t = tc.tiles3[blockIdx.x];
    const int ncols = 10 * B;
    const int N = (ncols + 15) / 16 * 16;
    const int nbc = N / 8;                      // column blocks
    const uint32_t tcols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
    const int T = d.T, J2 = d.J2;
    const int kjb = tc.kj / 8;
    tc_prologue(sm, tcols);

    int chunk = 0;
    for (int c0 = 0; c0 < kjb; c0 += kTcChunkKB, ++chunk) {
        const int kbc = min(kTcChunkKB, kjb - c0);
        const int kw = kbc * 8;                 // latitudes in this chunk
        const uint32_t abytes = static_cast<uint32_t>(t.nrb) * kbc * 128;
        if (threadIdx.x == 0) {
            expect_tx(&sm.mbar_ld, abytes * NP);
#pragma unroll
            for (int i = 0; i < NP; ++i)
                bulk_copy(sa + i * kAElems, tc.a3 + i * tc.elems3 + t.aoff + static_cast<long long>(t.nrb) * 64 * c0,
                          abytes, &sm.mbar_ld);
        }
        // zero the A row blocks beyond the tile's rows (not touched by the copy)
#pragma unroll
        for (int i = 0; i < NP; ++i) zero_range(sa + i * kAElems, t.nrb * kbc * 64, 16 * kbc * 64);
        // B = W^T chunk: [col block][kb][8 cols][8 latitudes]; loads issued in
        // batches of 8 independent requests per thread, then split and stored
        const int items = (N / 2) * kw;
        for (int base0 = 0; base0 < items; base0 += 8 * kTcThreads) {
            float2 wv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = base0 + u * kTcThreads + threadIdx.x;
                wv[u] = make_float2(0.f, 0.f);
                if (k < items) {
                    const int cp = k / kw, jj = k - cp * kw;
                    const int j = c0 * 8 + jj;
                    if (2 * cp < ncols && j < J2) {
                        const int b = cp / 5, g = cp - b * 5;
                        wv[u] = f2[((static_cast<size_t>(b) * (T + 1) + t.m) * 5 + g) * 2 * J2 + t.p * J2 + j];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = base0 + u * kTcThreads + threadIdx.x;
                if (k < items) {
                    const int cp = k / kw, jj = k - cp * kw;
                    const int c = 2 * cp;
                    const int e = ((c >> 3) * kbc + (jj >> 3)) * 64 + (c & 7) * 8 + (jj & 7);
                    split_store<NP>(wv[u].x, sb, kBElems, e);
                    split_store<NP>(wv[u].y, sb, kBElems, e + 8);   // column c + 1: next core row
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (!block_wait(sm, &sm.mbar_ld, chunk & 1, tc.err, 1)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (threadIdx.x == 0) {
            issue_chunk<NP>(sa, sb, sm.tmem, kbc, N, chunk == 0);
            mma_commit(&sm.mbar_mma);
        }
        if (!block_wait(sm, &sm.mbar_mma, chunk & 1, tc.err, 2)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
    }

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
// Columns col = b*8 + f*2 + (re, im) of the prepared coefficients
// C[q][col] (fields zeta, Phi', U, V as in the FP64/FP32 synthesis), read
// from cbuf[b][e][4] (FP32).  Output F1[b][j][f][p][m] (float2).
// ---------------------------------------------------------------------------
template <int NP>
__global__ void __launch_bounds__(kTcThreads) k1_tc(TcTables tc, Dims d, int B, const float2 *__restrict__ cbuf,
                                                    float2 *__restrict__ f1) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(smem_raw);
    __nv_bfloat16 *sa = a_base<NP>(smem_raw);
    __nv_bfloat16 *sb = b_base<NP>(smem_raw);
    const TcTile1 t = tc.tiles1[blockIdx.x];
    const int ncols = 8 * B;
    const int N = (ncols + 15) / 16 * 16;
    const int nbc = N / 8;
    const uint32_t tcols = N <= 32 ? 32u : 64u;
    const int T = d.T;
    const int m = t.m;
    const int krb = t.KR / 8;
    tc_prologue(sm, tcols);

    int chunk = 0;
    for (int c0 = 0; c0 < krb; c0 += kTcChunkKB, ++chunk) {
        const int kbc = min(kTcChunkKB, krb - c0);
        const int kw = kbc * 8;                 // rows q in this chunk
        const uint32_t abytes = static_cast<uint32_t>(t.njb) * kbc * 128;
        if (threadIdx.x == 0) {
            expect_tx(&sm.mbar_ld, abytes * NP);
#pragma unroll
            for (int i = 0; i < NP; ++i)
                bulk_copy(sa + i * kAElems, tc.a1 + i * tc.elems1 + t.aoff + static_cast<long long>(t.njb) * 64 * c0,
                          abytes, &sm.mbar_ld);
        }
#pragma unroll
        for (int i = 0; i < NP; ++i) zero_range(sa + i * kAElems, t.njb * kbc * 64, 16 * kbc * 64);
        // B = C^T chunk: [col block][kb][8 cols][8 rows q]; one column block
        // per state holds the 4 complex prepared coefficients of row q
        const int items = nbc * kw;
        for (int base0 = 0; base0 < items; base0 += 2 * kTcThreads) {
            float4 cv[2][2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int k = base0 + u * kTcThreads + threadIdx.x;
                cv[u][0] = cv[u][1] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < items) {
                    const int bb = k / kw, qq = k - bb * kw;
                    const int q = c0 * 8 + qq;
                    if (bb < B && q < t.R) {
                        const float4 *src = reinterpret_cast<const float4 *>(
                            cbuf + (static_cast<size_t>(bb) * d.next + ext_offset(T, m) + t.p + 2 * q) * 4);
                        cv[u][0] = src[0];
                        cv[u][1] = src[1];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int k = base0 + u * kTcThreads + threadIdx.x;
                if (k < items) {
                    const int bb = k / kw, qq = k - bb * kw;
                    const int e = (bb * kbc + (qq >> 3)) * 64 + (qq & 7);
                    split_store<NP>(cv[u][0].x, sb, kBElems, e + 0 * 8);
                    split_store<NP>(cv[u][0].y, sb, kBElems, e + 1 * 8);
                    split_store<NP>(cv[u][0].z, sb, kBElems, e + 2 * 8);
                    split_store<NP>(cv[u][0].w, sb, kBElems, e + 3 * 8);
                    split_store<NP>(cv[u][1].x, sb, kBElems, e + 4 * 8);
                    split_store<NP>(cv[u][1].y, sb, kBElems, e + 5 * 8);
                    split_store<NP>(cv[u][1].z, sb, kBElems, e + 6 * 8);
                    split_store<NP>(cv[u][1].w, sb, kBElems, e + 7 * 8);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (!block_wait(sm, &sm.mbar_ld, chunk & 1, tc.err, 3)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (threadIdx.x == 0) {
            issue_chunk<NP>(sa, sb, sm.tmem, kbc, N, chunk == 0);
            mma_commit(&sm.mbar_mma);
        }
        if (!block_wait(sm, &sm.mbar_mma, chunk & 1, tc.err, 4)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
    }

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

// Synthesis coefficients in FP32, one thread per (extended row e, state b):
// cbuf[b][e] = (zeta, Phi', U, V) of degree n' (the wind factors as in the
// FP64/FP32 synthesis), each state value converted once.
__global__ void k1_prep_f32(const double2 *__restrict__ states, long long sstride, Dims d,
                            const double *__restrict__ syn, const int *__restrict__ row_m, float2 *__restrict__ cbuf) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (e >= d.next) return;
    const int T = d.T, nc = d.ncoef;
    const int m = row_m[e];
    const int n = m + (e - ext_offset(T, m));
    const int off = order_offset(T, m);
    const double2 *st = states + b * sstride;
    auto ld = [&](int f, int k) -> double2 {
        return (k >= m && k <= T) ? st[f * nc + off + k - m] : make_double2(0.0, 0.0);
    };
    const double2 z0 = ld(F_ZETA, n), zm = ld(F_ZETA, n - 1), zp = ld(F_ZETA, n + 1);
    const double2 d0 = ld(F_DIV, n), dm = ld(F_DIV, n - 1), dp = ld(F_DIV, n + 1);
    const double2 p0 = ld(F_PHI, n);
    const double c0 = syn[3 * e], c1 = syn[3 * e + 1], c2 = syn[3 * e + 2];
    float4 *o = reinterpret_cast<float4 *>(cbuf + (static_cast<size_t>(b) * d.next + e) * 4);
    o[0] = make_float4(float(z0.x), float(z0.y), float(p0.x), float(p0.y));
    o[1] = make_float4(float(-c0 * d0.y - c1 * zm.x - c2 * zp.x), float(c0 * d0.x - c1 * zm.y - c2 * zp.y),
                       float(-c0 * z0.y + c1 * dm.x + c2 * dp.x), float(c0 * z0.x + c1 * dm.y + c2 * dp.y));
}

}  // namespace

cudaError_t configure_tc_kernels() {
    const int s2 = (int)tc_smem_bytes(2), s3 = (int)tc_smem_bytes(3);
    cudaError_t e = cudaFuncSetAttribute(k3_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k3_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, s3);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k1_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s2);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k1_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, s3);
    return e;
}

cudaError_t launch_tc_synthesis(const TcTables &tc, const Dims &d, int B, const double2 *states, long long sstride,
                                const double *syn, const int *row_m, float2 *cbuf, float2 *f1, cudaStream_t s) {
    if (B < 1 || B > kMaxNodes) return cudaErrorInvalidValue;
    k1_prep_f32<<<dim3((d.next + 127) / 128, B), 128, 0, s>>>(states, sstride, d, syn, row_m, cbuf);
    if (tc.npieces == 2) k1_tc<2><<<tc.ntiles1, kTcThreads, tc_smem_bytes(2), s>>>(tc, d, B, cbuf, f1);
    else k1_tc<3><<<tc.ntiles1, kTcThreads, tc_smem_bytes(3), s>>>(tc, d, B, cbuf, f1);
    return cudaGetLastError();
}

cudaError_t launch_tc_projection(const TcTables &tc, const Dims &d, int B, const float2 *f2, float2 *y,
                                 cudaStream_t s) {
    if (B < 1 || B > kMaxNodes) return cudaErrorInvalidValue;
    if (tc.npieces == 2) k3_tc<2><<<tc.ntiles3, kTcThreads, tc_smem_bytes(2), s>>>(tc, d, B, f2, y);
    else k3_tc<3><<<tc.ntiles3, kTcThreads, tc_smem_bytes(3), s>>>(tc, d, B, f2, y);
    return cudaGetLastError();
}

}  // namespace sdc
