// rt_born_tc.cu — the contractions of the ray-Born operator (arXiv:2511.18511
// Sec. 3.5 and the Appendix; Green's functions g_t = A_t exp(i omega T_t)):
//
//   apply    d[f][e][r] = w_f sum_{x in ring} E_e(x) E_r(x) dc(x),  e != r,
//   adjoint  dc~(x)     = Re sum_f w_f sum_{e != r} conj(E_e(x) E_r(x)) d[f][e][r],
//
// w_f = omega^2 h^2, E_t(x) = A_t(x) exp(-omega_s^y L_t(x)) exp(i 2 pi f T_t(x)),
// on the 5th-generation tensor cores (tcgen05, kind::tf32, accumulators in
// tensor memory) with FP32-level accuracy by a two-term TF32 split: every
// operand value v = hi + lo with hi = tf32(v), lo = tf32(v - hi), and a
// product is hi*hi + hi*lo + lo*hi (error ~2^-21 relative). The E field is
// never stored: producer warps form it from the T, A (and L) maps in the
// shared-memory operand layout of the MMA (K-major, 128-byte swizzle).
//
// Complex arithmetic as real GEMMs: the K axis interleaves real and imaginary
// parts, (Re, Im) of each node (apply) or of each receiver (adjoint).
//   apply, unit (f, tile (bi <= bj) of 128 x 128 transducers): A rows
//     e in bi: (Er, Ei); B rows r in bj: (Wr, -Wi) [real part], then
//     (Wi, Wr) [imaginary part], W = dc E; the 128 x 256 accumulator holds
//     Re and Im of sum_x E_e W_r. d is symmetric, so only bi <= bj is formed
//     (10 of 16 tiles for 512 transducers). The K axis (nodes) is cut into
//     chunks; items (chunk, unit) go round-robin to one block per SM, chunk-
//     major, so the blocks at work share the maps of two or three chunks in
//     L2; each item's partial sums are added with vector reductions.
//   adjoint, item (128 nodes, f): with D'[e][r] = conj(d[e][r] + d[r][e]) for
//     e < r (0 otherwise), sum_{e != r} conj(E_e E_r) d = conj(sum_e E_e
//     sum_{r > e} D'[e][r] E_r) up to the real part, so for each block of 128
//     e the accumulator V(x, e) = sum_r D'[e][r] E_r(x) (A rows x: (Er, Ei)
//     per r; B rows e: (D'r, -D'i) then (D'i, D'r)) runs over r-blocks >= the
//     e-block only, and the epilogue forms Re sum_e E_e(x) V(x, e) per node.
//     B (the D' tiles, pre-split and pre-swizzled by k_born_dprep, 64 KB per
//     16 receivers) is copied with bulk async copies and stays in L2.
//
// Block roles (one block per SM): warp 0 allocates tensor memory and one of
// its lanes issues the MMAs; warps 1-4 are the epilogue (warp w reads TMEM
// lanes 32 (w mod 4) ...); warps 5-12 produce the A (and, for the apply, B)
// stages; warp 13 (adjoint) issues the B copies. Two operand stages, two
// accumulators (2 x 256 TMEM columns) so the epilogue of one accumulation
// overlaps the next. Every wait is bounded (rt_tc.cuh): a stuck pipeline
// sets *err and the block tears down and frees its tensor memory.
//
// The FP32 SIMT path (RTBORN_GEMM_FP32) forms E and W in global memory
// (k_born_efield in rt_born.cu) and runs the hand-written complex GEMM
// k_cgemm below.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include <cuda_runtime.h>

#include "rt_internal.h"
#include "rt_tc.cuh"

namespace rt {

namespace {

using namespace tc;

constexpr int kRows = 128;                                 // MMA M, transducers per block
constexpr uint32_t kPlaneA = 128 * 128;                    // 128 rows x 128 B
constexpr uint32_t kPlaneB = 256 * 128;                    // 256 rows x 128 B
constexpr uint32_t kStageBytes = 2 * kPlaneA + 2 * kPlaneB;   // A hi, A lo, B hi, B lo: 96 KB
constexpr int kStages = 2;
constexpr int kEpiWarp0 = 1, kProdWarp0 = 5, kCopyWarp = 13;
constexpr int kProdThreads = 256;
constexpr int kApplyThreads = 13 * 32;
constexpr int kAdjThreads = 14 * 32;
constexpr uint32_t kTmemCols = 512;
constexpr int kBars = 9;   // full[2], empty[2], acc_full[2], acc_empty[2], drain
constexpr size_t kSmem = kStages * kStageBytes + 1024 + 128;
constexpr uint32_t kIdesc = idesc_tf32(128, 256);
constexpr int kErrApply = 101, kErrAdjoint = 102;
// K-tiles (16 nodes each) the apply accumulates in tensor memory before adding
// the partial sums to the global accumulator. The error of the tensor core's
// FP32 accumulation grows linearly with the number of MMAs summed into one
// accumulator (measured at full size, 1024^2 / 512-ring, against FP64 sums of
// the same maps: 2.2e-6 relative after runs of 8 K-tiles, 4.1e-6 after 16,
// 7.4e-6 after 32, 5.6e-5 after 256; the FP32 SIMT path: 3.4e-6), while the
// added reductions cost about 6 ms at 16 and 3 ms at 32.
constexpr int kApplyChunk = 16;

struct TCArgs {
    int n_tx, nb, n_tiles, n_freq, n_in;
    long long nn;                       // nodes per map
    const int* idx;                     // inside-ring nodes, padded to a multiple of 128 with node 0
    const float* T;
    const float* A;
    const float* L;                     // [n_tx][nn] maps (L only with absorption)
    const float* dc;                    // [nn] (apply)
    BornFreq fq[kBornFreqMax];
    int nk, chunk;                      // apply: K-tiles of 16 nodes, K-tiles per chunk
    long long n_items;
    float* acc;                         // apply: [n_freq * n_tiles][128][256]
    const float* bd;                    // adjoint: D' tiles [f][tile][8][2][256][32]
    float* part;                        // adjoint: [n_freq][n_in]
    int* err;
    int accumulate;                     // adjoint finish: add to the output
};

__device__ __forceinline__ void tile_rc(int tile, int nb, int* bi, int* bj) {
    int b = 0, rem = tile;
    while (rem >= nb - b) {
        rem -= nb - b;
        ++b;
    }
    *bi = b;
    *bj = b + rem;
}

// E = A exp(-wy L) exp(i 2 pi frac(f T)); 0 where T is unreached (+inf) or NaN.
// Branch-free, so that callers can issue all their map loads first.
template <bool LOSSY>
__device__ __forceinline__ float2 efield(float T, float A, float L, const BornFreq& f) {
    const bool ok = T < 3.0e38f;
    const float Tc = ok ? T : 0.f;
    const float pr = f.fh * Tc;                         // frac(f T), f = fh + fl, product error by FMA
    const float er = fmaf(f.fh, Tc, -pr);
    const float fr = (pr - rintf(pr)) + fmaf(f.fl, Tc, er);
    float sn, cs;
    __sincosf(6.28318530717958648f * fr, &sn, &cs);
    float a = ok ? A : 0.f;
    if (LOSSY) a *= __expf(-f.wy * (ok ? L : 0.f));
    return make_float2(a * cs, a * sn);
}

// hi/lo TF32 split of four values, stored at one 16-byte chunk of each plane
__device__ __forceinline__ void put_split(uint32_t hi_addr, uint32_t lo_addr, float a, float b, float c, float d) {
    const float ha = to_tf32(a), hb = to_tf32(b), hc = to_tf32(c), hd = to_tf32(d);
    st_shared_v4(hi_addr, ha, hb, hc, hd);
    st_shared_v4(lo_addr, to_tf32(a - ha), to_tf32(b - hb), to_tf32(c - hc), to_tf32(d - hd));
}

// byte offset of 16-byte chunk c of row m in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t swz(int m, int c) { return (uint32_t)m * 128u + (uint32_t)((c ^ (m & 7)) << 4); }

struct Smem {
    uint32_t base;          // 1024-aligned shared address of stage 0
    uint64_t* bars;
    uint32_t* tslot;
    volatile int* abort_flag;
};

__device__ __forceinline__ Smem carve(uint8_t* raw) {
    Smem s;
    const uint32_t r = smem_u32(raw);
    s.base = (r + 1023u) & ~1023u;
    uint8_t* g = raw + (s.base - r);
    s.bars = (uint64_t*)(g + kStages * kStageBytes);
    s.tslot = (uint32_t*)(s.bars + kBars);
    s.abort_flag = (volatile int*)(s.tslot + 1);
    return s;
}

__device__ __forceinline__ uint32_t bar_addr(const Smem& s, int i) { return smem_u32(s.bars + i); }

__device__ void setup(const Smem& S, uint32_t full_count) {
    if (threadIdx.x == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(bar_addr(S, st), full_count);
            mbar_init(bar_addr(S, 2 + st), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_addr(S, 4 + b), 1);
            mbar_init(bar_addr(S, 6 + b), 4);
        }
        mbar_init(bar_addr(S, 8), 1);
        *S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(S.tslot), kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
}

// MMA thread: drain every MMA it issued, then the block frees tensor memory.
__device__ void teardown(const Smem& S, uint32_t tmem, bool mma_thread, int* err, int code) {
    if (mma_thread) {
        mma_commit(bar_addr(S, 8));
        volatile int never = 0;   // the drain waits even after an abort
        mbar_wait(bar_addr(S, 8), 0, &never, err, code);
    }
    __syncwarp();
    fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after_sync();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Issues the 3 split products of one stage (4 K-steps of 8 TF32 columns).
__device__ __forceinline__ void mma_stage(uint32_t stage, uint32_t d_tmem, bool* first) {
    const uint32_t ah = stage, al = stage + kPlaneA, bh = stage + 2 * kPlaneA, bl = bh + kPlaneB;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint32_t ko = 32u * kk;
        const uint64_t dah = desc_sw128(ah + ko), dal = desc_sw128(al + ko);
        const uint64_t dbh = desc_sw128(bh + ko), dbl = desc_sw128(bl + ko);
        mma_tf32(d_tmem, dah, dbh, kIdesc, *first ? 0u : 1u);
        *first = false;
        mma_tf32(d_tmem, dah, dbl, kIdesc, 1u);
        mma_tf32(d_tmem, dal, dbh, kIdesc, 1u);
    }
}

// ---------------------------------------------------------------- apply

template <bool LOSSY>
__global__ void __launch_bounds__(kApplyThreads, 1) k_born_apply_tc(const __grid_constant__ TCArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const Smem S = carve(smem_raw);
    setup(S, kProdThreads / 32);
    const uint32_t tmem = *S.tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int U = a.n_freq * a.n_tiles;
    bool mma_thread = false;

    if (warp == 0) {
        if (lane == 0) {
            mma_thread = true;
            uint32_t q = 0, j = 0;
            for (long long it = blockIdx.x; it < a.n_items; it += gridDim.x, ++j) {
                const int c = (int)(it / U);
                const int kt0 = c * a.chunk, kt1 = min(kt0 + a.chunk, a.nk);
                const uint32_t b = j & 1;
                if (!mbar_wait(bar_addr(S, 6 + b), ((j >> 1) & 1) ^ 1, S.abort_flag, a.err, kErrApply)) break;
                fence_after_sync();
                const uint32_t d = tmem + b * 256;
                bool first = true, ok = true;
                for (int kt = kt0; kt < kt1; ++kt, ++q) {
                    const uint32_t st = q & 1;
                    if (!mbar_wait(bar_addr(S, st), (q >> 1) & 1, S.abort_flag, a.err, kErrApply)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    mma_stage(S.base + st * kStageBytes, d, &first);
                    mma_commit(bar_addr(S, 2 + st));
                }
                if (!ok) break;
                mma_commit(bar_addr(S, 4 + b));
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
        const int qtr = warp & 3, m = qtr * 32 + lane;
        uint32_t j = 0;
        for (long long it = blockIdx.x; it < a.n_items; it += gridDim.x, ++j) {
            const int u = (int)(it % U);
            const int f = u / a.n_tiles;
            int bi, bj;
            tile_rc(u - f * a.n_tiles, a.nb, &bi, &bj);
            const uint32_t b = j & 1;
            bool ok = mbar_wait(bar_addr(S, 4 + b), (j >> 1) & 1, S.abort_flag, a.err, kErrApply);
            if (!__all_sync(0xffffffffu, ok)) break;
            fence_after_sync();
            float* dst = a.acc + ((size_t)u * kRows + m) * 256;
            const bool row_ok = bi * kRows + m < a.n_tx;
            for (int cc = 0; cc < 8; ++cc) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(qtr * 32) << 16) + b * 256 + cc * 32, v);
                if (row_ok) {
#pragma unroll
                    for (int i = 0; i < 32; i += 4) red_add_v4(dst + cc * 32 + i, v[i], v[i + 1], v[i + 2], v[i + 3]);
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_addr(S, 6 + b));
        }
    } else if (warp >= kProdWarp0) {
        // a half-warp covers the 16 nodes of one K-tile for one transducer row,
        // so every map load of a warp reads two rows x 64 contiguous bytes.
        // Rows of this thread: A rows tA + 16 i and B rows tB + 16 i (i < 8).
        // All 16 (or 24) map values of a stage are loaded before any is used,
        // and those of the next stage while this one is formed.
        const int pw = warp - kProdWarp0, j = lane & 15, sub = lane >> 4;
        constexpr int NL = LOSSY ? 16 : 1;
        uint32_t q = 0;
        for (long long it = blockIdx.x; it < a.n_items; it += gridDim.x) {
            const int c = (int)(it / U), u = (int)(it % U);
            const int f = u / a.n_tiles;
            int bi, bj;
            tile_rc(u - f * a.n_tiles, a.nb, &bi, &bj);
            const BornFreq& fq = a.fq[f];
            const int tA = bi * kRows + 2 * pw + sub, tB = bj * kRows + 2 * pw + sub;
            const int kt0 = c * a.chunk, kt1 = min(kt0 + a.chunk, a.nk);
            float Tn[16], An[16], Ln[NL], wn;
            bool pvn;
            auto load = [&](int kt) {
                const int p = kt * 16 + j;
                pvn = p < a.n_in;
                const int k = a.idx[p];
                wn = a.dc[k];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int t = (i < 8 ? tA : tB) + 16 * (i & 7);
                    const bool v = pvn && t < a.n_tx;
                    const size_t o = (size_t)(v ? t : 0) * (size_t)a.nn + k;
                    Tn[i] = v ? a.T[o] : __uint_as_float(0x7f800000u);
                    An[i] = v ? a.A[o] : 0.f;
                    if (LOSSY) Ln[i & (NL - 1)] = v ? a.L[o] : 0.f;
                }
            };
            load(kt0);
            bool ok = true;
            for (int kt = kt0; kt < kt1; ++kt, ++q) {
                float Tc[16], Ac[16], Lc[NL];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    Tc[i] = Tn[i];
                    Ac[i] = An[i];
                    if (LOSSY) Lc[i & (NL - 1)] = Ln[i & (NL - 1)];
                }
                const float wdc = wn;
                if (kt + 1 < kt1) load(kt + 1);
                const uint32_t st = q & 1;
                ok = mbar_wait(bar_addr(S, 2 + st), ((q >> 1) & 1) ^ 1, S.abort_flag, a.err, kErrApply);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                const uint32_t sb = S.base + st * kStageBytes;
                const uint32_t cofs = (uint32_t)(j & 1) * 8u;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int m = 2 * pw + sub + 16 * (i & 7);
                    const float2 E = efield<LOSSY>(Tc[i], Ac[i], LOSSY ? Lc[i & (NL - 1)] : 0.f, fq);
                    const uint32_t off = swz(m, j >> 1) + cofs;
                    if (i < 8) {
                        const float hr = to_tf32(E.x), hi = to_tf32(E.y);
                        st_shared_v2(sb + off, hr, hi);
                        st_shared_v2(sb + kPlaneA + off, to_tf32(E.x - hr), to_tf32(E.y - hi));
                    } else {
                        const float wr = wdc * E.x, wi = wdc * E.y;
                        const float hr = to_tf32(wr), hi = to_tf32(wi);
                        const float lr = to_tf32(wr - hr), li = to_tf32(wi - hi);
                        const uint32_t bh = sb + 2 * kPlaneA, bl = bh + kPlaneB;
                        st_shared_v2(bh + off, hr, -hi);
                        st_shared_v2(bl + off, lr, -li);
                        st_shared_v2(bh + off + kRows * 128, hi, hr);
                        st_shared_v2(bl + off + kRows * 128, li, lr);
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_addr(S, st));
            }
            if (!ok) break;
        }
    }
    teardown(S, tmem, mma_thread, a.err, kErrApply);
}

// d[f][e][r] = w_f (acc_re + i acc_im) of the tile holding (min, max) of the
// two blocks, mirrored; 0 on the diagonal.
__global__ void k_born_apply_finish(const __grid_constant__ TCArgs a, float2* __restrict__ d) {
    const long long n = (long long)a.n_freq * a.n_tx * a.n_tx;
    const bool bad = *(volatile int*)a.err != 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(i / ((long long)a.n_tx * a.n_tx));
        const int rem = (int)(i - (long long)f * a.n_tx * a.n_tx);
        int e = rem / a.n_tx, r = rem - (rem / a.n_tx) * a.n_tx;
        if (e == r) {
            d[i] = make_float2(0.f, 0.f);
            continue;
        }
        if (e / kRows > r / kRows) {
            const int t = e;
            e = r;
            r = t;
        }
        const int bi = e / kRows, bj = r / kRows;
        const int tile = bi * a.nb - (bi * (bi - 1)) / 2 + (bj - bi);
        const float* s = a.acc + ((size_t)(f * a.n_tiles + tile) * kRows + (e % kRows)) * 256;
        const float w = bad ? __uint_as_float(0x7fc00000u) : a.fq[f].scale;
        d[i] = make_float2(w * s[r % kRows], w * s[128 + r % kRows]);
    }
}

// ---------------------------------------------------------------- adjoint

// D' tiles: [f][tile (be <= br)][kt (8)][plane (hi, lo)][256 rows][128 B],
// 128-byte-swizzled like the shared-memory B stage, one thread per 16-byte chunk.
__global__ void k_born_dprep(int n_tx, int nb, int n_tiles, int n_freq, const float2* __restrict__ d,
                             float* __restrict__ bd) {
    const long long n = (long long)n_freq * n_tiles * 8 * 256 * 8;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(g & 7), row = (int)((g >> 3) & 255), kt = (int)((g >> 11) & 7);
        const long long rest = g >> 14;
        const int tile = (int)(rest % n_tiles), f = (int)(rest / n_tiles);
        int be, br;
        tile_rc(tile, nb, &be, &br);
        const int e = be * kRows + (row & 127);
        const bool im = row >= 128;
        float v[4];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int r = br * kRows + kt * 16 + 2 * c + k;
            float2 D = make_float2(0.f, 0.f);
            if (e < r && r < n_tx) {
                const float2 a1 = d[((size_t)f * n_tx + e) * n_tx + r], a2 = d[((size_t)f * n_tx + r) * n_tx + e];
                D = make_float2(a1.x + a2.x, -(a1.y + a2.y));   // conj(d[e][r] + d[r][e])
            }
            v[2 * k] = im ? D.y : D.x;
            v[2 * k + 1] = im ? D.x : -D.y;
        }
        float* blk = bd + ((((size_t)f * n_tiles + tile) * 8 + kt) * 2) * 8192;
        const int off = row * 32 + ((c ^ (row & 7)) << 2);
        float hi[4], lo[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            hi[k] = to_tf32(v[k]);
            lo[k] = to_tf32(v[k] - hi[k]);
        }
        *(float4*)(blk + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *(float4*)(blk + 8192 + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
}

__device__ __forceinline__ int ktiles_of(int br, int n_tx) { return min(8, (n_tx - br * kRows + 15) / 16); }

template <bool LOSSY>
__global__ void __launch_bounds__(kAdjThreads, 1) k_born_adjoint_tc(const __grid_constant__ TCArgs a) {
    extern __shared__ uint8_t smem_raw[];
    const Smem S = carve(smem_raw);
    setup(S, kProdThreads / 32 + 1);
    const uint32_t tmem = *S.tslot;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    bool mma_thread = false;

    if (warp == 0) {
        if (lane == 0) {
            mma_thread = true;
            uint32_t q = 0, pc = 0;
            bool ok = true;
            for (long long it = blockIdx.x; ok && it < a.n_items; it += gridDim.x) {
                for (int be = 0; ok && be < a.nb; ++be, ++pc) {
                    const uint32_t b = pc & 1;
                    if (!(ok = mbar_wait(bar_addr(S, 6 + b), ((pc >> 1) & 1) ^ 1, S.abort_flag, a.err, kErrAdjoint)))
                        break;
                    fence_after_sync();
                    const uint32_t d = tmem + b * 256;
                    bool first = true;
                    for (int br = be; ok && br < a.nb; ++br) {
                        const int nkt = ktiles_of(br, a.n_tx);
                        for (int kt = 0; kt < nkt; ++kt, ++q) {
                            const uint32_t st = q & 1;
                            if (!(ok = mbar_wait(bar_addr(S, st), (q >> 1) & 1, S.abort_flag, a.err, kErrAdjoint)))
                                break;
                            fence_after_sync();
                            mma_stage(S.base + st * kStageBytes, d, &first);
                            mma_commit(bar_addr(S, 2 + st));
                        }
                    }
                    if (ok) mma_commit(bar_addr(S, 4 + b));
                }
            }
        }
        __syncwarp();
    } else if (warp == kCopyWarp) {
        if (lane == 0) {
            uint32_t q = 0;
            bool ok = true;
            for (long long it = blockIdx.x; ok && it < a.n_items; it += gridDim.x) {
                const int f = (int)(it % a.n_freq);
                for (int be = 0; ok && be < a.nb; ++be)
                    for (int br = be; ok && br < a.nb; ++br) {
                        const int tile = be * a.nb - (be * (be - 1)) / 2 + (br - be);
                        const int nkt = ktiles_of(br, a.n_tx);
                        for (int kt = 0; kt < nkt; ++kt, ++q) {
                            const uint32_t st = q & 1;
                            if (!(ok = mbar_wait(bar_addr(S, 2 + st), ((q >> 1) & 1) ^ 1, S.abort_flag, a.err,
                                                 kErrAdjoint)))
                                break;
                            const float* src = a.bd + ((((size_t)f * a.n_tiles + tile) * 8 + kt) * 2) * 8192;
                            mbar_arrive_tx(bar_addr(S, st), 2 * kPlaneB);
                            bulk_g2s(S.base + st * kStageBytes + 2 * kPlaneA, src, 2 * kPlaneB, bar_addr(S, st));
                        }
                    }
            }
        }
        __syncwarp();
    } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4) {
        // Re sum_e E_e(x) V(x, e) in groups of 16 e: the maps of a group are
        // loaded before the accumulator is read, those of the next group
        // while this one is summed.
        const int qtr = warp & 3, m = qtr * 32 + lane;
        constexpr int NL = LOSSY ? 16 : 1;
        uint32_t pc = 0;
        bool ok = true;
        for (long long it = blockIdx.x; ok && it < a.n_items; it += gridDim.x) {
            const int xb = (int)(it / a.n_freq), f = (int)(it % a.n_freq);
            const int x = xb * kRows + m;
            const bool xv = x < a.n_in;
            const int k = a.idx[x];
            const BornFreq& fq = a.fq[f];
            float sacc = 0.f;
            float Tn[16], An[16], Ln[NL];
            auto load = [&](int e0) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = e0 + i;
                    const bool v = xv && e < a.n_tx;
                    const size_t o = (size_t)(v ? e : 0) * (size_t)a.nn + k;
                    Tn[i] = v ? a.T[o] : __uint_as_float(0x7f800000u);
                    An[i] = v ? a.A[o] : 0.f;
                    if (LOSSY) Ln[i & (NL - 1)] = v ? a.L[o] : 0.f;
                }
            };
            for (int be = 0; be < a.nb; ++be, ++pc) {
                load(be * kRows);
                const uint32_t b = pc & 1;
                ok = mbar_wait(bar_addr(S, 4 + b), (pc >> 1) & 1, S.abort_flag, a.err, kErrAdjoint);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                fence_after_sync();
                const uint32_t ta = tmem + ((uint32_t)(qtr * 32) << 16) + b * 256;
                for (int g = 0; g < 8; ++g) {
                    float Tc[16], Ac[16], Lc[NL];
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        Tc[i] = Tn[i];
                        Ac[i] = An[i];
                        if (LOSSY) Lc[i & (NL - 1)] = Ln[i & (NL - 1)];
                    }
                    if (g + 1 < 8) load(be * kRows + 16 * (g + 1));
                    float vr[16], vi[16];
                    tmem_ld16(ta + 16 * g, vr);
                    tmem_ld16(ta + 128 + 16 * g, vi);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float2 E = efield<LOSSY>(Tc[i], Ac[i], LOSSY ? Lc[i & (NL - 1)] : 0.f, fq);
                        sacc = fmaf(E.x, vr[i], fmaf(-E.y, vi[i], sacc));
                    }
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_addr(S, 6 + b));
            }
            if (ok && xv) a.part[(size_t)f * a.n_in + x] = sacc;
        }
    } else if (warp >= kProdWarp0 && warp < kProdWarp0 + 8) {
        // thread: node row m of the A tile, receivers r0 .. r0 + 7 of each
        // stage (r0 = br 128 + kt 16 + 8 hf); map values of the next stage are
        // loaded while this one is formed
        const int pt = threadIdx.x - kProdWarp0 * 32;
        const int m = pt & 127, hf = pt >> 7;
        constexpr int NL = LOSSY ? 8 : 1;
        uint32_t q = 0;
        bool ok = true;
        for (long long it = blockIdx.x; ok && it < a.n_items; it += gridDim.x) {
            const int xb = (int)(it / a.n_freq), f = (int)(it % a.n_freq);
            const int x = xb * kRows + m;
            const bool xv = x < a.n_in;
            const int k = a.idx[x];
            const BornFreq& fq = a.fq[f];
            float Tn[8], An[8], Ln[NL];
            auto load = [&](int r0) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = r0 + i;
                    const bool v = xv && r < a.n_tx;
                    const size_t o = (size_t)(v ? r : 0) * (size_t)a.nn + k;
                    Tn[i] = v ? a.T[o] : __uint_as_float(0x7f800000u);
                    An[i] = v ? a.A[o] : 0.f;
                    if (LOSSY) Ln[i & (NL - 1)] = v ? a.L[o] : 0.f;
                }
            };
            // stages of the item in order: (be, br >= be, kt < ktiles_of(br))
            int be = 0, br = 0, kt = 0;
            load(8 * hf);
            while (ok && be < a.nb) {
                int nbe = be, nbr = br, nkt = kt + 1;
                if (nkt >= ktiles_of(br, a.n_tx)) {
                    nkt = 0;
                    if (++nbr >= a.nb) nbr = ++nbe;
                }
                float Tc[8], Ac[8], Lc[NL];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    Tc[i] = Tn[i];
                    Ac[i] = An[i];
                    if (LOSSY) Lc[i & (NL - 1)] = Ln[i & (NL - 1)];
                }
                if (nbe < a.nb) load(nbr * kRows + nkt * 16 + 8 * hf);
                const uint32_t st = q & 1;
                ok = mbar_wait(bar_addr(S, 2 + st), ((q >> 1) & 1) ^ 1, S.abort_flag, a.err, kErrAdjoint);
                if (!(ok = __all_sync(0xffffffffu, ok))) break;
                const uint32_t sb = S.base + st * kStageBytes;
#pragma unroll
                for (int cl = 0; cl < 4; ++cl) {
                    const float2 E0 = efield<LOSSY>(Tc[2 * cl], Ac[2 * cl], LOSSY ? Lc[(2 * cl) & (NL - 1)] : 0.f, fq);
                    const float2 E1 =
                        efield<LOSSY>(Tc[2 * cl + 1], Ac[2 * cl + 1], LOSSY ? Lc[(2 * cl + 1) & (NL - 1)] : 0.f, fq);
                    const int ch = 4 * hf + cl;
                    put_split(sb + swz(m, ch), sb + kPlaneA + swz(m, ch), E0.x, E0.y, E1.x, E1.y);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_addr(S, st));
                ++q;
                be = nbe;
                br = nbr;
                kt = nkt;
            }
        }
    }
    teardown(S, tmem, mma_thread, a.err, kErrAdjoint);
}

// dc~(idx[p]) (+)= sum_f w_f part[f][p], summed in FP64; NaN after an expired wait
__global__ void k_born_adjoint_finish(const __grid_constant__ TCArgs a, float* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.n_in) return;
    double s = 0.0;
    for (int f = 0; f < a.n_freq; ++f) s += (double)a.fq[f].scale * (double)a.part[(size_t)f * a.n_in + p];
    if (*(volatile int*)a.err != 0) s = __longlong_as_double(0x7ff8000000000000ll);
    const int k = a.idx[p];
    out[k] = a.accumulate ? (float)((double)out[k] + s) : (float)s;
}

// ------------------------------------------------------- FP32 SIMT complex GEMM

// C(m, n) += sum_k A(m, k) B(n, k) over this block's K-range (blockIdx.z of
// gridDim.z equal slices), complex64, element (m, k) of A at A[m*sam + k*sak],
// likewise B and C; 64 x 64 outputs per block of 256 threads (4 x 4 each),
// K-steps of 16 staged in shared memory; C pre-zeroed, partial sums added
// atomically. AK / BK: the operand is contiguous along k (else along m / n),
// which sets the coalesced load order.
template <bool AK, bool BK>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int K, const float2* __restrict__ A, long long sam,
                                               long long sak, const float2* __restrict__ B, long long sbn,
                                               long long sbk, float2* __restrict__ C, long long scm, long long scn) {
    __shared__ float2 As[16][65], Bs[16][65];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int kslice = (K + gridDim.z - 1) / gridDim.z;
    const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            const int e = threadIdx.x + 256 * l;       // 1024 elements of each 64 x 16 tile
            const int kk = AK ? (e & 15) : (e >> 6), mm = AK ? (e >> 4) : (e & 63);
            const int k = k0 + kk, m = m0 + mm;
            As[kk][mm] = (k < ke && m < M) ? A[m * sam + k * sak] : make_float2(0.f, 0.f);
            const int kb2 = BK ? (e & 15) : (e >> 6), nn = BK ? (e >> 4) : (e & 63);
            const int k2 = k0 + kb2, n = n0 + nn;
            Bs[kb2][nn] = (k2 < ke && n < N) ? B[n * sbn + k2 * sbk] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float2 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(av[i].x, bv[j].x, fmaf(-av[i].y, bv[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(av[i].x, bv[j].y, fmaf(av[i].y, bv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty * 4 + i, n = n0 + tx * 4 + j;
            if (m < M && n < N) {
                float2* c = C + m * scm + n * scn;
                atomicAdd(&c->x, acc[i][j].x);
                atomicAdd(&c->y, acc[i][j].y);
            }
        }
}

int sm_count(int device) {
    static std::atomic<int> cache[64];
    if (device < 0 || device >= 64) return 152;
    int v = cache[device].load(std::memory_order_relaxed);
    if (!v) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 152;
        cache[device].store(v, std::memory_order_relaxed);
    }
    return v;
}

}  // namespace

size_t born_tc_acc_bytes(int n_tx, int n_freq) {
    const int nb = (n_tx + kRows - 1) / kRows;
    return sizeof(float) * (size_t)n_freq * (size_t)(nb * (nb + 1) / 2) * kRows * 256;
}

size_t born_tc_bd_bytes(int n_tx, int n_freq) {
    const int nb = (n_tx + kRows - 1) / kRows;
    return (size_t)n_freq * (size_t)(nb * (nb + 1) / 2) * 8 * 2 * kPlaneB;
}

cudaError_t launch_born_apply_tc(int device, const BornTCJob& j, float* acc, float2* d, int* err, cudaStream_t s) {
    TCArgs a{};
    a.n_tx = j.n_tx;
    a.nb = (j.n_tx + kRows - 1) / kRows;
    a.n_tiles = a.nb * (a.nb + 1) / 2;
    a.n_freq = j.n_freq;
    a.n_in = j.n_in;
    a.nn = j.nn;
    a.idx = j.idx;
    a.T = j.T;
    a.A = j.A;
    a.L = j.L;
    a.dc = j.dc;
    for (int f = 0; f < j.n_freq && f < kBornFreqMax; ++f) a.fq[f] = j.fq[f];
    a.acc = acc;
    a.err = err;
    a.nk = (j.n_in + 15) / 16;
    const int G = sm_count(device);
    const long long U = (long long)a.n_freq * a.n_tiles;
    a.chunk = j.chunk > 0 ? j.chunk : kApplyChunk;
    a.n_items = ((a.nk + a.chunk - 1) / a.chunk) * U;
    cudaError_t e = cudaMemsetAsync(acc, 0, born_tc_acc_bytes(j.n_tx, j.n_freq), s);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(G, a.n_items));
    if (j.L) {
        e = cudaFuncSetAttribute(k_born_apply_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess) k_born_apply_tc<true><<<grid, kApplyThreads, kSmem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_born_apply_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess) k_born_apply_tc<false><<<grid, kApplyThreads, kSmem, s>>>(a);
    }
    if (e != cudaSuccess) return e;
    const long long n = (long long)a.n_freq * a.n_tx * a.n_tx;
    k_born_apply_finish<<<(unsigned)std::min<long long>((n + 255) / 256, 4096), 256, 0, s>>>(a, d);
    return cudaGetLastError();
}

cudaError_t launch_born_adjoint_tc(int device, const BornTCJob& j, const float2* d, float* bd, float* part,
                                   float* dc_out, bool accumulate, int* err, cudaStream_t s) {
    TCArgs a{};
    a.n_tx = j.n_tx;
    a.nb = (j.n_tx + kRows - 1) / kRows;
    a.n_tiles = a.nb * (a.nb + 1) / 2;
    a.n_freq = j.n_freq;
    a.n_in = j.n_in;
    a.nn = j.nn;
    a.idx = j.idx;
    a.T = j.T;
    a.A = j.A;
    a.L = j.L;
    for (int f = 0; f < j.n_freq && f < kBornFreqMax; ++f) a.fq[f] = j.fq[f];
    a.bd = bd;
    a.part = part;
    a.err = err;
    a.accumulate = accumulate ? 1 : 0;
    a.n_items = (long long)((j.n_in + kRows - 1) / kRows) * a.n_freq;
    const long long nprep = (long long)a.n_freq * a.n_tiles * 8 * 256 * 8;
    k_born_dprep<<<(unsigned)std::min<long long>((nprep + 255) / 256, 8192), 256, 0, s>>>(a.n_tx, a.nb, a.n_tiles,
                                                                                            a.n_freq, d, bd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int G = sm_count(device);
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(G, a.n_items));
    if (j.L) {
        e = cudaFuncSetAttribute(k_born_adjoint_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess) k_born_adjoint_tc<true><<<grid, kAdjThreads, kSmem, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_born_adjoint_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e == cudaSuccess) k_born_adjoint_tc<false><<<grid, kAdjThreads, kSmem, s>>>(a);
    }
    if (e != cudaSuccess) return e;
    k_born_adjoint_finish<<<(j.n_in + 255) / 256, 256, 0, s>>>(a, dc_out);
    return cudaGetLastError();
}

cudaError_t launch_cgemm(int M, int N, int K, const float2* A, long long sam, long long sak, const float2* B,
                         long long sbn, long long sbk, float2* C, long long scm, long long scn, int device,
                         cudaStream_t s) {
    const dim3 blk(256);
    const unsigned gx = (M + 63) / 64, gy = (N + 63) / 64;
    const int G = sm_count(device);
    // split K until the grid covers the GPU about four times over
    const long long base = (long long)gx * gy;
    const unsigned gz = (unsigned)std::max<long long>(1, std::min<long long>((4LL * G * 4 + base - 1) / base,
                                                                            std::max(1, K / 256)));
    const dim3 grid(gx, gy, gz);
    const bool ak = sak == 1, bk = sbk == 1;
    if (ak && bk) k_cgemm<true, true><<<grid, blk, 0, s>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, scm, scn);
    else if (ak) k_cgemm<true, false><<<grid, blk, 0, s>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, scm, scn);
    else if (bk) k_cgemm<false, true><<<grid, blk, 0, s>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, scm, scn);
    else k_cgemm<false, false><<<grid, blk, 0, s>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, scm, scn);
    return cudaGetLastError();
}

}  // namespace rt
