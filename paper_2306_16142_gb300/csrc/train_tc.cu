// Tensor-core training path of the BF16 working copy (Sec. 5.1: the DDF network is optimised
// with Adam on the loss of its two outputs). Every contraction of the forward and reverse
// passes is a tcgen05 BF16 GEMM with FP32 accumulators in tensor memory, fed by TMA:
//
//   forward  a_{l+1} = ReLU(a_l W_l^T + b_l)          A = a_l      [m][K_l]   B = W_l   [W][K_l]
//   head     y = a_L W_out^T + b_out, the loss, G = dLoss/dy and
//            delta_{L-1} = (G W_out) * 1[a_L > 0]
//   dgrad    delta_{l-1} = (delta_l W_l) * 1[a_l > 0] A = delta_l  [m][W]     B = W_l^T [K_l][W]
//   wgrad    dW_l = delta_l^T a_l                     A = delta_l^T [W][m]    B = a_l^T [K_l][m]
//            (K = the batch: split over CTAs, partials summed in a fixed order)
//
// For widths 128 / 256 with K0 <= 128 the step runs as fused persistent kernels: the forward on
// tile pairs (the query's pair kernel in its training form; the loss form of the two-output head
// folded into its last layer), the data-gradient chain on tile pairs (mlp_pairb_kernel, every
// delta kept on chip as the next step's A operand), all layers' weight gradients in one launch
// (wgrad_all_kernel, which also takes the deltas' column sums, the bias gradients, from its
// operand stages), their split sums (wsum_all_kernel), the fixed-order bias-gradient stages and
// one launch for the loss, Adam and the repacking (adam_pack_kernel). Other shapes use the one
// persistent GEMM kernel below for every contraction: per CTA a TMA producer warp, an MMA warp
// (one thread issues M = 128, N = BN, K = 16 MMAs into one of two TMEM accumulators, so a tile's
// epilogue overlaps the next tile's MMAs) and eight epilogue warps (two column halves x four TMEM
// lane quadrants; thread = row). Either way activations and deltas are written once, row-major
// BF16: the forward / dgrad read them K-major, and the wgrad reads the same arrays as MN-major
// operands (its K is the batch), so no transposed copy is ever made. ReLU masks are kept as bits;
// every gradient sum is a fixed-order reduction of partials, so a step is bit-reproducible.
#include <math.h>

#include <algorithm>

#include "ddf_internal.cuh"
#include "device_common.cuh"
#include "tc_common.cuh"

namespace ddf {
namespace {

constexpr int kTEpi = 8;                       // epilogue warps
constexpr int kTThreads = (kTEpi + 2) * 32;    // + TMA producer warp + MMA warp
constexpr uint32_t kSmemMax = 232448;          // 227 KB of dynamic shared memory per CTA

enum { T_FWD = 0, T_DGRAD = 2, T_WGRAD = 3, T_STORE = 4 };

struct TArgs {
    int mode;
    int M, N, BN;             // A has M rows, B has N rows; BN: N per tile (64..256, multiple of 64)
    int nkb, kb_per, ksplit;  // K-blocks (64 wide) in total and per split; number of splits
    int b_layer;              // third coordinate of B's tensor map
    int nst;                  // pipeline stages
    int mn_major;             // operands are MN-major (wgrad: A and B read from row-major [K][MN])
    int bres;                 // B (the weights, N == BN) loaded once per CTA and kept in shared memory
    uint32_t off_stage, off_blk, off_bias, off_bar;
    const float* bias;        // [N]
    __nv_bfloat16* out;       // [rows][N]
    uint32_t* mask_out;       // [rows][N / 32] (nullable)
    const uint32_t* mask_in;  // [rows][N / 32]
    float* colpart;           // [rows / 32][N]
    float* fout;              // T_WGRAD: [ksplit][M][N]; T_STORE: [rows][N]
    int* err;
};

// A warp's 32 x 32 BF16 block lives in 2 KB of shared memory: 32 lines of 64 B, the four 16-byte
// pieces of line l stored at piece ^ ((l >> 1) & 3), so that eight consecutive lines written at
// one logical piece, and two consecutive lines read whole, both touch every bank once. Reads go
// four lanes to a line (lane: line 8 i + lane / 4, piece lane % 4), so every global store
// instruction writes eight 64-byte segments: whole sectors, each written once.
__device__ __forceinline__ uint32_t blk_off(int line, int piece) {
    return (uint32_t)(line * 64 + 16 * (piece ^ ((line >> 1) & 3)));
}

// line = this lane's row (row-major staging of the lane's 32 values)
__device__ __forceinline__ void stage_rows(uint8_t* tb, int lane, const uint32_t pk[16]) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
        *reinterpret_cast<uint4*>(tb + blk_off(lane, p)) =
            make_uint4(pk[4 * p], pk[4 * p + 1], pk[4 * p + 2], pk[4 * p + 3]);
    __syncwarp();
}

// Piece (lane % 4) of line (8 i + lane / 4).
__device__ __forceinline__ uint4 blk_read(const uint8_t* tb, int lane, int i) {
    return *reinterpret_cast<const uint4*>(tb + blk_off(8 * i + (lane >> 2), lane & 3));
}

// Rows row0..row0+31 (lane = row) of columns col0..col0+31 to a row-major [.][ld] array.
// colsum (nullable) gets each column's sum over the 32 rows of the BF16 values: every lane sums
// its piece's 8 columns over its 4 rows, then the 8 lanes holding one piece combine in a fixed
// butterfly.
__device__ __forceinline__ void store_rows(uint8_t* tb, int lane, const uint32_t pk[16], __nv_bfloat16* out,
                                           int64_t ld, int64_t row0, int col0, float* colsum) {
    stage_rows(tb, lane, pk);
    float cs[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) cs[e] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint4 v = blk_read(tb, lane, i);
        *reinterpret_cast<uint4*>(out + (row0 + 8 * i + (lane >> 2)) * ld + col0 + 8 * (lane & 3)) = v;
        if (colsum) {
            cs[0] += bf_lo(v.x); cs[1] += bf_hi(v.x);
            cs[2] += bf_lo(v.y); cs[3] += bf_hi(v.y);
            cs[4] += bf_lo(v.z); cs[5] += bf_hi(v.z);
            cs[6] += bf_lo(v.w); cs[7] += bf_hi(v.w);
        }
    }
    if (colsum) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float t = cs[e];
            t += __shfl_xor_sync(0xffffffffu, t, 4);
            t += __shfl_xor_sync(0xffffffffu, t, 8);
            t += __shfl_xor_sync(0xffffffffu, t, 16);
            cs[e] = t;
        }
        if (lane < 4) {
            float4* dst = reinterpret_cast<float4*>(colsum + col0 + 8 * lane);
            dst[0] = make_float4(cs[0], cs[1], cs[2], cs[3]);
            dst[1] = make_float4(cs[4], cs[5], cs[6], cs[7]);
        }
    }
    __syncwarp();
}

// MN-major operand with 128-byte swizzle: rows of 64 MN elements (128 B), one row per K index;
// 8-row K groups 1024 B apart (SBO), 64-wide MN atoms 8 KB apart (LBO: one 64 x 64 TMA box).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(8192 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__global__ void __launch_bounds__(kTThreads, 1)
    train_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                      const TArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NST = a.nst, BN = a.BN, N = a.N;
    const uint32_t stage_bytes = 16384u + (a.bres ? 0u : (uint32_t)BN * 128u);
    uint8_t* bres = smem;                    // resident B: K-block kb at kb * BN * 128
    uint8_t* stages = smem + a.off_stage;
    uint8_t* blk = smem + a.off_blk;
    float* bias_s = reinterpret_cast<float*>(smem + a.off_bias);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + a.off_bar);
    uint64_t* full = bars;
    uint64_t* empty = bars + NST;
    uint64_t* accf = bars + 2 * NST;
    uint64_t* acce = accf + 2;
    uint64_t* bfull = acce + 2;  // resident B loaded
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bfull + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntm = (a.M + 127) / 128, ntn = N / BN;
    const int64_t ntiles = (int64_t)ntm * ntn * a.ksplit;
    const uint32_t tcols = BN <= 128 ? 256u : 512u;

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accf[0], 1);
        mbar_init(&accf[1], 1);
        mbar_init(&acce[0], kTEpi * 32);
        mbar_init(&acce[1], kTEpi * 32);
        mbar_init(bfull, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (a.mode == T_FWD)
        for (int i = tid; i < N; i += kTThreads) bias_s[i] = a.bias[i];
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    // Launched as a programmatic dependent of the previous kernel in the stream: the set-up above
    // (and the resident weights, which no kernel of the step writes) overlaps its tail; nothing
    // it produced is read, and nothing it reads is written, before this wait.
    if (a.bres && tid == kTEpi * 32) {
        mbar_expect_tx(bfull, (uint32_t)a.nkb * (uint32_t)BN * 128u);
        for (int kb = 0; kb < a.nkb; ++kb)
            tma_load_3d(bres + (size_t)kb * BN * 128, &mapB, bfull, kb * 64, 0, a.b_layer);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (warp == kTEpi) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t cnt = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int s = (int)(t / (ntm * ntn)), rem = (int)(t % (ntm * ntn));
                const int tm = rem % ntm, tn = rem / ntm;
                const int kb0 = s * a.kb_per, kb1 = min(a.nkb, kb0 + a.kb_per);
                for (int kb = kb0; kb < kb1; ++kb, ++cnt) {
                    const int stg = (int)(cnt % (uint32_t)NST);
                    const uint32_t ph = (cnt / (uint32_t)NST) & 1u;
                    if (!mbar_wait(&empty[stg], ph ^ 1u, a.err)) { ok = false; break; }
                    uint8_t* sa = stages + (size_t)stg * stage_bytes;
                    mbar_expect_tx(&full[stg], stage_bytes);
                    if (a.bres) {
                        tma_load_3d(sa, &mapA, &full[stg], kb * 64, tm * 128, 0);
                    } else if (a.mn_major) {
                        // 64 x 64 boxes of the row-major [K][MN] arrays, 8 KB apart
                        for (int j = 0; j < 2; ++j)
                            tma_load_3d(sa + j * 8192, &mapA, &full[stg], tm * 128 + 64 * j, kb * 64, 0);
                        for (int j = 0; j < BN / 64; ++j)
                            tma_load_3d(sa + 16384 + j * 8192, &mapB, &full[stg], tn * BN + 64 * j, kb * 64, 0);
                    } else {
                        tma_load_3d(sa, &mapA, &full[stg], kb * 64, tm * 128, 0);
                        tma_load_3d(sa + 16384, &mapB, &full[stg], kb * 64, tn * BN, a.b_layer);
                    }
                }
            }
        }
    } else if (warp == kTEpi + 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t cnt = 0, tl = 0;
            bool ok = true;
            // MN-major operands: bits 15 / 16 of the instruction descriptor
            const uint32_t idesc = idesc_bf16(128, BN) | (a.mn_major ? (3u << 15) : 0u);
            if (a.bres && !mbar_wait(bfull, 0u, a.err)) ok = false;
            for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
                const int s = (int)(t / (ntm * ntn));
                const int kb0 = s * a.kb_per, kb1 = min(a.nkb, kb0 + a.kb_per);
                const uint32_t buf = tl & 1u;
                if (!mbar_wait(&acce[buf], ((tl >> 1) & 1u) ^ 1u, a.err)) break;
                tc_fence_after();
                const uint32_t d = tbase + buf * (uint32_t)BN;
                for (int kb = kb0; kb < kb1; ++kb, ++cnt) {
                    const int stg = (int)(cnt % (uint32_t)NST);
                    const uint32_t ph = (cnt / (uint32_t)NST) & 1u;
                    if (!mbar_wait(&full[stg], ph, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(stages + (size_t)stg * stage_bytes);
                    if (a.bres) {
                        const uint64_t ad = sdesc(sa), bd = sdesc(su32(bres) + (uint32_t)kb * (uint32_t)BN * 128u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) mma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (kb > kb0 || k > 0));
                    } else if (a.mn_major) {
                        // K step of 16 rows = two 1024-byte swizzle atoms
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_bf16(d, sdesc_mn(sa + 2048u * k), sdesc_mn(sa + 16384u + 2048u * k), idesc,
                                     (kb > kb0 || k > 0));
                    } else {
                        const uint64_t ad = sdesc(sa), bd = sdesc(sa + 16384u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) mma_bf16(d, ad + 2 * k, bd + 2 * k, idesc, (kb > kb0 || k > 0));
                    }
                    mma_commit(&empty[stg]);
                }
                if (ok) mma_commit(&accf[buf]);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int grp = warp >> 2, q = warp & 3;
        const int r = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        uint8_t* tb = blk + warp * 2048;
        const int nhalf = BN / 64;             // 32-column chunks per column group (1..4)
        const int ch0 = grp * nhalf;
        const int NW = N / 32;
        uint32_t tl = 0;
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
            const int s = (int)(t / (ntm * ntn)), rem = (int)(t % (ntm * ntn));
            const int tm = rem % ntm, tn = rem / ntm;
            const uint32_t buf = tl & 1u;
            const int64_t row = (int64_t)tm * 128 + r;
            const int64_t wrow0 = (int64_t)tm * 128 + q * 32;   // first row of this warp
            const int64_t rblk = (int64_t)tm * 4 + q;           // 32-row block index
            uint32_t mwords[4] = {0u, 0u, 0u, 0u};
            if (a.mode == T_DGRAD) {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                    if (cc < nhalf) mwords[cc] = a.mask_in[row * NW + (tn * BN) / 32 + ch0 + cc];
            }
            if (!mbar_wait(&accf[buf], (tl >> 1) & 1u, a.err)) break;
            tc_fence_after();
            const uint32_t tacc = tbase + lane_off + buf * (uint32_t)BN;

            if (a.mode == T_FWD || a.mode == T_DGRAD) {
                // chunks in pairs: two TMEM loads behind one wait
                auto chunk = [&](int cc, const uint32_t* raw) {
                    const int col0 = tn * BN + (ch0 + cc) * 32;
                    uint32_t pk[16];
                    if (a.mode == T_FWD) {
                        uint32_t bits = 0;
                        const float4* b4 = reinterpret_cast<const float4*>(bias_s + col0);
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4) {
                            const float4 b = b4[j4];
                            float x0, x1, x2, x3;
                            add2(__uint_as_float(raw[4 * j4]), __uint_as_float(raw[4 * j4 + 1]), b.x, b.y, x0, x1);
                            add2(__uint_as_float(raw[4 * j4 + 2]), __uint_as_float(raw[4 * j4 + 3]), b.z, b.w, x2, x3);
                            bits |= (pos(x0) << (4 * j4)) | (pos(x1) << (4 * j4 + 1)) | (pos(x2) << (4 * j4 + 2)) |
                                    (pos(x3) << (4 * j4 + 3));
                            pk[2 * j4] = pack_relu(x0, x1);
                            pk[2 * j4 + 1] = pack_relu(x2, x3);
                        }
                        mwords[cc] = bits;
                    } else {
                        const uint32_t bits = mwords[cc];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float x0 = (bits >> (2 * j)) & 1u ? __uint_as_float(raw[2 * j]) : 0.f;
                            const float x1 = (bits >> (2 * j + 1)) & 1u ? __uint_as_float(raw[2 * j + 1]) : 0.f;
                            pk[j] = pack_bf16(x0, x1);
                        }
                    }
                    store_rows(tb, lane, pk, a.out, N, wrow0, col0,
                               a.mode == T_DGRAD ? a.colpart + rblk * N : nullptr);
                };
#pragma unroll
                for (int cc = 0; cc < 4; cc += 2) {
                    if (cc >= nhalf) break;
                    uint32_t r0[32], r1[32];
                    TC_LD32(tacc + (ch0 + cc) * 32, r0);
                    if (cc + 1 < nhalf) TC_LD32(tacc + (ch0 + cc + 1) * 32, r1);
                    tc_wait_ld();
                    chunk(cc, r0);
                    if (cc + 1 < nhalf) chunk(cc + 1, r1);
                }
                if (a.mode == T_FWD && a.mask_out) {
                    uint32_t* mo = a.mask_out + row * NW + (tn * BN) / 32 + ch0;
                    if (nhalf == 4)
                        *reinterpret_cast<uint4*>(mo) = make_uint4(mwords[0], mwords[1], mwords[2], mwords[3]);
                    else
                        for (int cc = 0; cc < nhalf; ++cc) mo[cc] = mwords[cc];
                }
            } else if (a.mode == T_WGRAD) {
                // fragment order: each store instruction writes 512 contiguous bytes
                float* base = a.fout + ((((int64_t)s * ntm + tm) * 4 + q) * (BN / 32)) * 1024;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    if (cc >= nhalf) break;
                    const int c = ch0 + cc;
                    uint32_t raw[32];
                    TC_LD32(tacc + c * 32, raw);
                    tc_wait_ld();
                    float4* dst = reinterpret_cast<float4*>(base + (int64_t)c * 1024) + lane;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        dst[32 * i] = make_float4(__uint_as_float(raw[4 * i]), __uint_as_float(raw[4 * i + 1]),
                                                  __uint_as_float(raw[4 * i + 2]), __uint_as_float(raw[4 * i + 3]));
                }
            } else if (a.mode == T_STORE) {
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    if (cc >= nhalf) break;
                    const int c = ch0 + cc;
                    uint32_t raw[32];
                    TC_LD32(tacc + c * 32, raw);
                    tc_wait_ld();
                    float4* dst = reinterpret_cast<float4*>(a.fout + row * N + tn * BN + c * 32);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        dst[i] = make_float4(__uint_as_float(raw[4 * i]), __uint_as_float(raw[4 * i + 1]),
                                             __uint_as_float(raw[4 * i + 2]), __uint_as_float(raw[4 * i + 3]));
                }
            }
            tc_fence_before();
            mbar_arrive(&acce[buf]);
        }
    }
    __syncthreads();
    if (*(volatile int*)a.err) {
        // error path: let MMAs and TMA copies already issued drain (they wait on nothing)
        const uint64_t t0 = gtimer();
        while (gtimer() - t0 < 200000ull) {
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tcols));
    }
}

// All layers' weight gradients of a chunk in one launch: work item = (layer l, split s of the
// batch rows); each CTA accumulates the whole dW_l = delta_l^T a_l (W x N_l, the 128-row halves in
// two TMEM accumulators) over its split, so every delta and activation K-block is read once, and
// writes it as one split-K partial slab in wsum_kernel's fragment order. Both operands are read
// MN-major from the row-major workspace arrays (64 x 64 TMA boxes), as in the per-layer wgrad.
// While the MMAs run, the epilogue warps take the column sums of every delta K-block from the
// same stages (the bias gradients db_l = sum over rows of delta_l): thread (cc, rg) owns the eight
// features [8 cc, 8 cc + 8) and the row group rg of each 64-row stage, rows in order, and writes
// its sums of the split once: bsum[l][s][rg][W] (W / 8 x rg_count threads, rg_count = 2048 / W).
struct WArgs {
    int L, W, K0, nst;
    int ks, kb_per, nkb;   // splits per layer, K-blocks (64 rows) per split, K-blocks in all
    uint32_t off_bar;
    float* part;           // layer l: ks slabs of W x N_l floats at part + l * ks * W * max(K0, W)
    float* bsum;           // [L][ks][2048 / W][W] column-sum partials of the deltas
    int* err;
};

__global__ void __launch_bounds__(kTThreads, 1)
    wgrad_all_kernel(const __grid_constant__ CUtensorMap mapD, const __grid_constant__ CUtensorMap mapA0,
                     const __grid_constant__ CUtensorMap mapAct, const WArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int NST = a.nst, W = a.W, KM = a.K0 > a.W ? a.K0 : a.W;
    const uint32_t a_bytes = (uint32_t)W * 128u;                 // delta K-block: W features x 64 rows
    const uint32_t stage_bytes = a_bytes + (uint32_t)KM * 128u;   // + activation K-block
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + a.off_bar);
    uint64_t* full = bars;
    uint64_t* empty = bars + NST;
    uint64_t* accf = bars + 2 * NST;
    uint64_t* acce = accf + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(acce + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t items = (int64_t)a.L * a.ks;
    const int nhalf = W / 128;   // M-halves of dW
    const uint32_t tcols = nhalf == 2 ? 512u : 256u;

    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1 + kTEpi);   // the MMA commit and every epilogue warp
        }
        mbar_init(accf, 1);
        mbar_init(acce, kTEpi * 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    // launched as a programmatic dependent of the data-gradient chain: nothing it wrote is read
    // before this wait
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    auto item_range = [&](int64_t t, int& l, int& s, int& n, int& kb0, int& kb1) {
        l = (int)(t / a.ks);
        s = (int)(t % a.ks);
        n = l == 0 ? a.K0 : W;
        kb0 = s * a.kb_per;
        kb1 = min(a.nkb, kb0 + a.kb_per);
    };

    if (warp == kTEpi) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            uint32_t stg = 0, ring_ph = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < items && ok; t += gridDim.x) {
                int l, s, n, kb0, kb1;
                item_range(t, l, s, n, kb0, kb1);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&empty[stg], ring_ph ^ 1u, a.err)) { ok = false; break; }
                    uint8_t* sa = smem + (size_t)stg * stage_bytes;
                    mbar_expect_tx(&full[stg], a_bytes + (uint32_t)n * 128u);
                    for (int j = 0; j < W / 64; ++j) tma_load_3d(sa + j * 8192, &mapD, &full[stg], 64 * j, kb * 64, l);
                    for (int j = 0; j < n / 64; ++j)
                        tma_load_3d(sa + a_bytes + j * 8192, l == 0 ? &mapA0 : &mapAct, &full[stg], 64 * j, kb * 64,
                                    l == 0 ? 0 : l - 1);
                    if (++stg == (uint32_t)NST) {
                        stg = 0;
                        ring_ph ^= 1u;
                    }
                }
            }
        }
    } else if (warp == kTEpi + 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t stg = 0, ring_ph = 0, tl = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < items && ok; t += gridDim.x, ++tl) {
                int l, s, n, kb0, kb1;
                item_range(t, l, s, n, kb0, kb1);
                const uint32_t idesc = idesc_bf16(128, n) | (3u << 15);   // both operands MN-major
                if (!mbar_wait(acce, (tl & 1u) ^ 1u, a.err)) break;       // the previous item is read
                tc_fence_after();
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!mbar_wait(&full[stg], ring_ph, a.err)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = su32(smem + (size_t)stg * stage_bytes);
                    for (int h = 0; h < nhalf; ++h)
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            mma_bf16(tbase + (uint32_t)h * 256u, sdesc_mn(sa + (uint32_t)h * 16384u + 2048u * k),
                                     sdesc_mn(sa + a_bytes + 2048u * k), idesc, (kb > kb0 || k > 0));
                    mma_commit(&empty[stg]);
                    if (++stg == (uint32_t)NST) {
                        stg = 0;
                        ring_ph ^= 1u;
                    }
                }
                if (ok) mma_commit(accf);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // warp w: M-half w / 4 (rows 128 h + 32 (w % 4) + lane of dW_l), every 32-column chunk
        const int h = warp >> 2, q = warp & 3;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        // column sums: thread (cc, rg), features [8 cc, 8 cc + 8) = 16-byte chunk cc % 8 of the
        // 64-feature box cc / 8, rows [rpg rg, rpg rg + rpg) of every stage
        const int ncc = W / 8, rgc = kTEpi * 32 / ncc, rpg = 64 / rgc;
        const int cc = tid % ncc, rg = tid / ncc;
        const uint32_t cbox = (uint32_t)(cc >> 3) * 8192u, cch = (uint32_t)(cc & 7);
        uint32_t tl = 0, stg = 0, ring_ph = 0;
        for (int64_t t = blockIdx.x; t < items; t += gridDim.x, ++tl) {
            int l, s, n, kb0, kb1;
            item_range(t, l, s, n, kb0, kb1);
            float cs[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) cs[e] = 0.f;
            bool ok = true;
            for (int kb = kb0; kb < kb1; ++kb) {
                ok = mbar_wait(&full[stg], ring_ph, a.err);
                if (!__all_sync(0xffffffffu, ok)) { ok = false; break; }
                const uint32_t sa = su32(smem + (size_t)stg * stage_bytes) + cbox;
                for (int i = 0; i < rpg; ++i) {
                    const int r = rg * rpg + i;
                    uint32_t v[4];
                    ld_shared_v4(sa + (uint32_t)r * 128u + ((cch ^ (uint32_t)(r & 7)) << 4), v);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        add2(cs[2 * e], cs[2 * e + 1], __uint_as_float(v[e] << 16),
                             __uint_as_float(v[e] & 0xffff0000u), cs[2 * e], cs[2 * e + 1]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[stg]);
                if (++stg == (uint32_t)NST) {
                    stg = 0;
                    ring_ph ^= 1u;
                }
            }
            if (!ok) break;
            {
                float4* dst = reinterpret_cast<float4*>(a.bsum + (((int64_t)l * a.ks + s) * rgc + rg) * W + 8 * cc);
                dst[0] = make_float4(cs[0], cs[1], cs[2], cs[3]);
                dst[1] = make_float4(cs[4], cs[5], cs[6], cs[7]);
            }
            if (!mbar_wait(accf, tl & 1u, a.err)) break;
            tc_fence_after();
            if (h < nhalf) {
                float* base = a.part + (int64_t)l * a.ks * W * KM + (int64_t)s * W * n +
                              ((int64_t)(h * 4 + q) * (n / 32)) * 1024;
                for (int c = 0; c < n / 32; ++c) {
                    uint32_t raw[32];
                    TC_LD32(tbase + lane_off + (uint32_t)h * 256u + (uint32_t)c * 32u, raw);
                    tc_wait_ld();
                    float4* dst = reinterpret_cast<float4*>(base + (int64_t)c * 1024) + lane;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        dst[32 * i] = make_float4(__uint_as_float(raw[4 * i]), __uint_as_float(raw[4 * i + 1]),
                                                  __uint_as_float(raw[4 * i + 2]), __uint_as_float(raw[4 * i + 3]));
                }
            }
            tc_fence_before();
            mbar_arrive(acce);
        }
    }
    __syncthreads();
    if (*(volatile int*)a.err) {
        const uint64_t t0 = gtimer();
        while (gtimer() - t0 < 200000ull) {
        }
        __syncthreads();
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(tcols));
    }
}

// Rows of the batch encoded in the tensor-core feature order (six raw coordinates, two zero
// columns, then per octave the sines and cosines), BF16, row-major [mp][K0]; rows m..mp-1 are
// zero.
__global__ void tenc_kernel(const float* __restrict__ o, const float* __restrict__ w, int64_t m, int64_t mp,
                            int E, int K0, __nv_bfloat16* __restrict__ X) {
    // one thread per row. sin / cos of 2^k pi v for k >= 1 by the double-angle recurrence seeded
    // by sincospi(v) (about 2^k ulp, far below the BF16 rounding that follows); exact for the
    // v whose sin / cos are 0 or +-1
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= mp) return;
    float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < m)
        for (int j = 0; j < 3; ++j) {
            v[j] = o[3 * r + j];
            v[3 + j] = w[3 * r + j];
        }
    const int noct = (E - 6) / 12;
    uint4* dst = reinterpret_cast<uint4*>(X + r * K0);
    float sn[6], cs[6];
    for (int j = 0; j < 6; ++j) sincospif(v[j], &sn[j], &cs[j]);
    dst[0] = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), 0u);
    int q = 1;   // next 16-byte chunk; octave k fills chunks 1 + 1.5 k .. (12 features)
    uint32_t pend[6];
    int np = 0;
    for (int k = 0; k < noct; ++k) {
        const float f[12] = {sn[0], sn[1], sn[2], sn[3], sn[4], sn[5], cs[0], cs[1], cs[2], cs[3], cs[4], cs[5]};
        for (int i = 0; i < 6; ++i) {
            pend[np++] = r < m ? pack_bf16(f[2 * i], f[2 * i + 1]) : 0u;
            if (np == 4) {
                dst[q++] = make_uint4(pend[0], pend[1], pend[2], pend[3]);
                np = 0;
            }
        }
        for (int j = 0; j < 6; ++j) {
            const float s2 = 2.f * sn[j] * cs[j];
            const float c2 = (cs[j] - sn[j]) * (cs[j] + sn[j]);
            sn[j] = s2;
            cs[j] = c2;
        }
    }
    while (np != 0 && np < 4) pend[np++] = 0u;
    if (np == 4) dst[q++] = make_uint4(pend[0], pend[1], pend[2], pend[3]);
    for (; q < K0 / 8; ++q) dst[q] = make_uint4(0u, 0u, 0u, 0u);
}

// dW_l (blob layout, [W][in]) += the split-K partials summed in split order. Partials are in the
// wgrad epilogue's fragment order (per split: M-tile, lane quadrant, 32-column chunk, float4
// index, lane); layer 0's internal columns are scattered back to the encoding order and its pad
// columns dropped.
__device__ __forceinline__ void wsum_block(const float4* __restrict__ part, int ksplit, int M, int N, int in_dim,
                                           int layer0, float* __restrict__ gW) {
    // block (32, 8): x = one float4 of the slab, y = a lane over the splits (y, y + 8, ...)
    const int64_t t = blockIdx.x * 32 + threadIdx.x;
    const int64_t slab4 = (int64_t)M * N / 4;
    __shared__ float4 red[8][32];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < slab4)
        for (int k = threadIdx.y; k < ksplit; k += 8) {
            const float4 v = part[(int64_t)k * slab4 + t];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y != 0 || t >= slab4) return;
    for (int k = 1; k < 8; ++k) {
        const float4 v = red[k][threadIdx.x];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    const int nch = N / 32;
    const int lane = (int)(t & 31), i = (int)((t >> 5) & 7);
    const int64_t u = t >> 8;
    const int c = (int)(u % nch), q = (int)((u / nch) & 3), tm = (int)(u / (nch * 4));
    const int o = tm * 128 + q * 32 + lane;
    const float vals[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int p = c * 32 + 4 * i + e;
        const int src = layer0 ? in_feature(p) : p;
        if (src >= 0 && src < in_dim) gW[(int64_t)o * in_dim + src] += vals[e];
    }
}

__global__ void wsum_kernel(const float4* __restrict__ part, int ksplit, int M, int N, int in_dim, int layer0,
                            float* __restrict__ gW) {
    wsum_block(part, ksplit, M, N, in_dim, layer0, gW);
}

// The split sums of every layer's weight gradient at once (blockIdx.y = layer; layer l's ks slabs
// of W x N_l floats at part + l * ks * W * KM, in the fragment order of the weight-gradient
// epilogue). Block (32, 8) takes one 32 x 32 piece of dW_l: thread (x, y) sums fragment float4
// (lane x, index y) over the splits in split order, the piece is transposed through shared
// memory, and each warp adds whole 32-column row segments to the gradient.
__global__ void wsum_all_kernel(const float4* __restrict__ part, int ks, int KM, int K0, NetLayout lay,
                                float* __restrict__ grad) {
    pdl_trigger();
    pdl_wait();
    const int l = blockIdx.y, W = lay.width;
    const int N = l == 0 ? K0 : W, nch = N / 32;
    const int u = blockIdx.x;   // (M-tile, lane quadrant, 32-column chunk) of the fragment order
    if (u >= (W / 32) * nch) return;
    const int x = threadIdx.x, y = threadIdx.y;
    const float4* P = part + (int64_t)l * ks * W * KM / 4;
    const int64_t slab4 = (int64_t)W * N / 4, t = (int64_t)u * 256 + y * 32 + x;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < ks; ++k) {
        const float4 v = P[k * slab4 + t];
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
    }
    __shared__ float piece[32][33];   // [row (lane)][column]
    piece[x][4 * y] = acc.x;
    piece[x][4 * y + 1] = acc.y;
    piece[x][4 * y + 2] = acc.z;
    piece[x][4 * y + 3] = acc.w;
    __syncthreads();
    const int c = u % nch, q = (u / nch) & 3, tm = u / (nch * 4);
    const int in_dim = l == 0 ? lay.E : W;
    float* gW = grad + lay.w_off[l];
    const int p = c * 32 + x;
    const int src = l == 0 ? in_feature(p) : p;
    if (src < 0 || src >= in_dim) return;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
        const int row = y + 8 * rr;
        gW[(int64_t)(tm * 128 + q * 32 + row) * in_dim + src] += piece[row][x];
    }
}

// Bias gradients db_l (blockIdx.y = l < L, from lrows partial column sums of delta_l, layer l's at
// lpart + l lstride) and the output layer's dW_out / db_out (blockIdx.y = L, from the hrows head
// partials), in two fixed-order stages: kBGroups groups of the partial rows (block (32, 8): 32
// consecutive outputs x 8 row lanes), then the groups in order.
constexpr int kBGroups = 16;
__global__ void bgrad_partial_kernel(const float* __restrict__ lpart, int64_t lrows, int64_t lstride,
                                     const float* __restrict__ headpart, int64_t hrows, NetLayout lay,
                                     float* __restrict__ bpart) {
    pdl_trigger();
    pdl_wait();
    const int l = blockIdx.y, g = blockIdx.z, W = lay.width;
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int ncol = l < lay.L ? W : 2 * W + 2;
    const int64_t ld = l < lay.L ? W : 2 * W + 2;
    const float* P = l < lay.L ? lpart + (int64_t)l * lstride : headpart;
    const int64_t nrb = l < lay.L ? lrows : hrows;
    const int64_t per = (nrb + kBGroups - 1) / kBGroups;
    const int64_t b0 = g * per, b1 = min(nrb, b0 + per);
    __shared__ float red[8][33];
    float s = 0.f;
    if (c < ncol)
        for (int64_t b = b0 + threadIdx.y; b < b1; b += 8) s += P[b * ld + c];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < ncol) {
        float t = red[0][threadIdx.x];
        for (int k = 1; k < 8; ++k) t += red[k][threadIdx.x];
        bpart[((int64_t)l * kBGroups + g) * (2 * W + 2) + c] = t;
    }
}

__global__ void bgrad_final_kernel(const float* __restrict__ bpart, NetLayout lay, float* __restrict__ grad) {
    pdl_trigger();
    pdl_wait();
    const int l = blockIdx.y, W = lay.width;
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int ncol = l < lay.L ? W : 2 * W + 2;
    if (c >= ncol) return;
    float t = 0.f;
    for (int g = 0; g < kBGroups; ++g) t += bpart[((int64_t)l * kBGroups + g) * (2 * W + 2) + c];
    float* out = l < lay.L ? grad + lay.b_off[l] + c
                           : (c < 2 * W ? grad + lay.w_off[lay.L] + c : grad + lay.b_off[lay.L] + (c - 2 * W));
    *out += t;
}

// d/d(o, w) from the gradient of the internal first-layer inputs gx [mp][K0].
__global__ void tenc_backward_kernel(const float* __restrict__ o, const float* __restrict__ w, int64_t m, int E,
                                     int K0, const float* __restrict__ gx, float* __restrict__ gin) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= m) return;
    float v[6];
    for (int j = 0; j < 3; ++j) {
        v[j] = o[3 * r + j];
        v[3 + j] = w[3 * r + j];
    }
    float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int p = 0; p < K0; ++p) {
        const int f = in_feature(p);
        if (f < 0 || f >= E) continue;
        const int j = f < 6 ? f : (f - 6) % 6;
        g[j] += gx[r * K0 + p] * encode_dfeature(f, v);
    }
    for (int j = 0; j < 6; ++j) gin[6 * r + j] = g[j];
}

// The output layer on the stored last activation a_L (row-major BF16 [mp][W], Sec. 4.1's
// two-output head): y = a_L W_out^T + b_out; the per-row loss terms and G = dLoss/dy (L1 on hit
// rows + BCE with logits; or the caller's cotangents); delta_{L-1} = (G W_out) * 1[a_L > 0],
// row-major BF16; and per-32-row partial sums of delta (db_{L-1}), of G a_L (dW_out) and of G
// (db_out). One warp per 32 rows; lane l owns columns [CPL l, CPL l + CPL) with CPL = W / 32.
struct HeadArgs {
    const __nv_bfloat16* aL;
    const float* head;        // W_out [2][W], b_out [2]
    __nv_bfloat16* delta;     // [mp][W]
    float* colpart;           // [mp / 32][W]
    float* headpart;          // [mp / 32][2W + 2]
    int64_t m, mp;
    const float* dist_gt;     // loss form
    const uint8_t* hit_gt;
    const int* n_hit;
    int64_t n_total;
    float* row_l1;
    float* row_bce;
    double* lossp;            // loss form, optional: per 32-row block (sum of L1 terms, sum of BCE terms)
    const float* gd_in;       // cotangent form
    const float* gl_in;
    int head_kind;            // DDF_HEAD_* (loss form)
    float head_delta;
};

// One lane's chunk of a BF16 row: CPL consecutive columns (CPL = 8: 16 bytes, CPL = 4: 8 bytes).
template <int CPL>
struct RowChunk {
    uint32_t u[CPL / 2];
    __device__ __forceinline__ void load(const __nv_bfloat16* p) {
        if constexpr (CPL == 8) {
            const uint4 v = *reinterpret_cast<const uint4*>(p);
            u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
        } else {
            const uint2 v = *reinterpret_cast<const uint2*>(p);
            u[0] = v.x; u[1] = v.y;
        }
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < CPL / 2; ++k) u[k] = 0u;
    }
    __device__ __forceinline__ void store(__nv_bfloat16* p) const {
        if constexpr (CPL == 8) *reinterpret_cast<uint4*>(p) = make_uint4(u[0], u[1], u[2], u[3]);
        else *reinterpret_cast<uint2*>(p) = make_uint2(u[0], u[1]);
    }
    __device__ __forceinline__ float at(int e) const { return (e & 1) ? bf_hi(u[e >> 1]) : bf_lo(u[e >> 1]); }
};

// v[0..31] of every lane -> v[0] of lane l holds the sum over the 32 lanes of v[l] (recursive
// halving: each step a lane keeps the half of its values whose index bit matches its lane bit and
// adds its partner's copy of that half; fixed order).
__device__ __forceinline__ void transpose_reduce32(float* v, int lane) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        const bool up = (lane & k) != 0;
#pragma unroll
        for (int m = 0; m < k; ++m) {
            const float send = up ? v[m] : v[m + k];
            const float keep = up ? v[m + k] : v[m];
            v[m] = keep + __shfl_xor_sync(0xffffffffu, send, k);
        }
    }
}

template <int W>
__global__ void __launch_bounds__(128, 4) head_kernel(const HeadArgs h) {
    constexpr int CPL = W / 32;
    const int lane = threadIdx.x & 31;
    const int64_t rblk = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (rblk * 32 >= h.mp) return;
    const int64_t row0 = rblk * 32;
    const int c0 = CPL * lane;
    float wo0[CPL], wo1[CPL];
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
        wo0[e] = h.head[c0 + e];
        wo1[e] = h.head[W + c0 + e];
    }
    // y of the 32 rows: each lane's CPL-column dot products, then summed across the lanes so that
    // lane i ends with row row0 + i
    float p0[32], p1[32];
#pragma unroll
    for (int i0 = 0; i0 < 32; i0 += 4) {
        RowChunk<CPL> ch[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (row0 + i0 + t < h.m) ch[t].load(h.aL + (row0 + i0 + t) * W + c0);
            else ch[t].zero();
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int e = 0; e < CPL; ++e) {
                s0 = fmaf(ch[t].at(e), wo0[e], s0);
                s1 = fmaf(ch[t].at(e), wo1[e], s1);
            }
            p0[i0 + t] = s0;
            p1[i0 + t] = s1;
        }
    }
    transpose_reduce32(p0, lane);
    transpose_reduce32(p1, lane);
    // lane i: the loss terms and G = dLoss/dy of row row0 + i
    const int64_t row = row0 + lane;
    float gd = 0.f, gl = 0.f, l1v = 0.f, bcev = 0.f;
    if (row < h.m) {
        const float d = p0[0] + h.head[2 * W], z = p1[0] + h.head[2 * W + 1];
        if (h.hit_gt) {
            const int nh = *h.n_hit;
            const float inv_h = nh > 0 ? 1.f / (float)nh : 0.f;
            const float inv_n = 1.f / (float)h.n_total;
            const bool hit = h.hit_gt[row] != 0;
            const float dg = hit ? h.dist_gt[row] : 0.f;
            if (h.head_kind != DDF_HEAD_TWO) {   // single output: y~ only (Eqs. 5, 7)
                single_head_loss(h.head_kind, h.head_delta, d, hit, dg, inv_n, &bcev, &gd);
            } else {
                const float lb = hit ? 1.f : 0.f;
                if (hit) {
                    const float diff = d - dg;
                    l1v = fabsf(diff);
                    gd = (diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f)) * inv_h;
                }
                gl = (1.f / (1.f + expf(-z)) - lb) * inv_n;
                bcev = fmaxf(z, 0.f) - z * lb + log1pf(expf(-fabsf(z)));
            }
            h.row_l1[row] = l1v;
            h.row_bce[row] = bcev;
        } else {
            gd = h.gd_in ? h.gd_in[row] : 0.f;
            gl = h.gl_in ? h.gl_in[row] : 0.f;
        }
    }
    if (h.lossp) {   // the block's loss terms by a fixed butterfly
        double s1 = l1v, s2 = bcev;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            h.lossp[2 * rblk] = s1;
            h.lossp[2 * rblk + 1] = s2;
        }
    }
    // db_out partial: the 32 rows' G by a fixed butterfly
    float sg0 = gd, sg1 = gl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sg0 += __shfl_xor_sync(0xffffffffu, sg0, o);
        sg1 += __shfl_xor_sync(0xffffffffu, sg1, o);
    }
    // delta_{L-1} = (G W_out) * 1[a_L > 0] row by row (512 contiguous bytes per warp store), its
    // column sums and the column sums of G a_L, rows in order
    float cd[CPL], cw0[CPL], cw1[CPL];
#pragma unroll
    for (int e = 0; e < CPL; ++e) cd[e] = cw0[e] = cw1[e] = 0.f;
#pragma unroll
    for (int i0 = 0; i0 < 32; i0 += 8) {
        RowChunk<CPL> ch[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            if (row0 + i0 + t < h.m) ch[t].load(h.aL + (row0 + i0 + t) * W + c0);
            else ch[t].zero();
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const float g0 = __shfl_sync(0xffffffffu, gd, i0 + t);
            const float g1 = __shfl_sync(0xffffffffu, gl, i0 + t);
            RowChunk<CPL> dl;
#pragma unroll
            for (int k = 0; k < CPL / 2; ++k) {
                const float a0 = ch[t].at(2 * k), a1 = ch[t].at(2 * k + 1);
                const float d0 = a0 > 0.f ? fmaf(g0, wo0[2 * k], g1 * wo1[2 * k]) : 0.f;
                const float d1 = a1 > 0.f ? fmaf(g0, wo0[2 * k + 1], g1 * wo1[2 * k + 1]) : 0.f;
                dl.u[k] = pack_bf16(d0, d1);
                cd[2 * k] += bf_lo(dl.u[k]);
                cd[2 * k + 1] += bf_hi(dl.u[k]);
                fma2p(g0, g0, a0, a1, cw0[2 * k], cw0[2 * k + 1], cw0[2 * k], cw0[2 * k + 1]);
                fma2p(g1, g1, a0, a1, cw1[2 * k], cw1[2 * k + 1], cw1[2 * k], cw1[2 * k + 1]);
            }
            dl.store(h.delta + (row0 + i0 + t) * W + c0);
        }
    }
    float* cp = h.colpart + rblk * W + c0;
    float* hp = h.headpart + rblk * (2 * W + 2);
#pragma unroll
    for (int e = 0; e < CPL; ++e) {
        cp[e] = cd[e];
        hp[c0 + e] = cw0[e];
        hp[W + c0 + e] = cw1[e];
    }
    if (lane == 0) {
        hp[2 * W] = sg0;
        hp[2 * W + 1] = sg1;
    }
}

// ------------------------------------------------------------------ host side
struct TLayout {
    uint32_t off_stage, off_blk, off_bias, off_bar, total;
    int nst;
};

// Shared memory: [resident B][stage ring][epilogue blocks][bias][barriers].
// Shared memory of the GEMM kernel: resident B (optional), the stages, the epilogue's staging
// blocks, the forward's bias of all N columns (at least 1 KB) and the barriers.
TLayout tlayout(int BN, int N, uint32_t bres_bytes) {
    TLayout s;
    const uint32_t stage = 16384u + (bres_bytes ? 0u : (uint32_t)BN * 128u);
    const uint32_t bias = std::max(1024u, (uint32_t)N * 4u);
    const uint32_t fixed = kTEpi * 2048 + bias + 256;
    const uint32_t avail = kSmemMax - 1024u - fixed - bres_bytes;
    s.nst = (int)std::min<uint32_t>(8u, avail / stage);
    uint32_t off = bres_bytes;
    s.off_stage = off; off += (uint32_t)s.nst * stage;
    s.off_blk = off;  off += kTEpi * 2048;
    s.off_bias = off; off += bias;
    s.off_bar = off;  off += 256;
    s.total = off + 1024;
    return s;
}

// BF16 3-D tensor map: `inner` elements per row (row stride `ld` elements), `rows` rows per
// slice, `depth` slices (slice stride rows * ld); box 64 x box_rows x 1, 128-byte swizzle.
int tmap(CUtensorMap* m, const void* base, uint64_t inner, uint64_t ld, uint64_t rows, uint64_t depth,
         uint32_t box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {inner, rows, depth};
    cuuint64_t strides[2] = {ld * 2, ld * rows * 2};
    cuuint32_t box[3] = {64, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DDF_OK;
}

int launch_gemm(const CUtensorMap& mA, const CUtensorMap& mB, TArgs a, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        DDF_CUDA_TRY(cudaFuncSetAttribute(train_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        attr = true;
    }
    if (a.BN % 64 || a.BN > 256 || a.N % a.BN) return fail(DDF_ERR_UNSUPPORTED, "training GEMM tile N=%d", a.BN);
    // weights as B (a single N tile): keep all of B in shared memory when it fits beside 2 A stages
    const uint32_t bres_bytes = (uint32_t)a.nkb * (uint32_t)a.BN * 128u;
    a.bres = (!a.mn_major && a.N == a.BN && a.ksplit == 1 && tlayout(a.BN, a.N, bres_bytes).nst >= 2) ? 1 : 0;
    const TLayout L = tlayout(a.BN, a.N, a.bres ? bres_bytes : 0u);
    if (L.nst < 2 || L.total > kSmemMax) return fail(DDF_ERR_UNSUPPORTED, "training GEMM shared memory");
    a.nst = L.nst;
    a.off_stage = L.off_stage;
    a.off_blk = L.off_blk;
    a.off_bias = L.off_bias;
    a.off_bar = L.off_bar;
    const int64_t ntiles = (int64_t)((a.M + 127) / 128) * (a.N / a.BN) * a.ksplit;
    const int grid = (int)std::min<int64_t>(ntiles, num_sms());
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kTThreads);
    cfg.dynamicSmemBytes = L.total;
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    DDF_CUDA_TRY(cudaLaunchKernelEx(&cfg, train_gemm_kernel, mA, mB, a));
    return DDF_OK;
}

// BF16 3-D tensor map of `depth` workspace arrays of `slice_rows` rows (row stride `inner`
// elements) of which the first `rows` are read (the rest as zero); box 64 x box_rows x 1,
// 128-byte swizzle.
int tmap_rows(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t slice_rows, uint64_t depth,
              uint32_t box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {inner, rows, depth};
    cuuint64_t strides[2] = {inner * 2, inner * slice_rows * 2};
    cuuint32_t box[3] = {64, box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(DDF_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DDF_OK;
}

// wgrad_all_kernel over rows [0, m) of the workspace arrays (row stride ld): deltas [L][ld][W],
// a_0 [ld][K0], a_1 .. a_{L-1} [L - 1][ld][W]; the partial slabs into part, the deltas' column-sum
// partials into bsum ([L][ks][2048 / W][W]). Returns the splits per layer.
int launch_wgrad_all(const ddf_net_s* net, const __nv_bfloat16* deltas, const __nv_bfloat16* a0,
                     const __nv_bfloat16* act1, int64_t m, int64_t ld, float* part, float* bsum, int* ks_out,
                     cudaStream_t s) {
    const NetLayout& lay = net->lay;
    const int W = lay.width, L = lay.L, K0 = net->tc->K0, KM = std::max(K0, W);
    CUtensorMap mD, mA0, mAct;
    int rc;
    if ((rc = tmap_rows(&mD, deltas, W, m, ld, L, 64))) return rc;
    if ((rc = tmap_rows(&mA0, a0, K0, m, ld, 1, 64))) return rc;
    if ((rc = tmap_rows(&mAct, act1, W, m, ld, std::max(1, L - 1), 64))) return rc;
    WArgs a{};
    a.L = L;
    a.W = W;
    a.K0 = K0;
    a.nkb = (int)((m + 63) / 64);
    const int want = std::max(1, std::min(a.nkb, num_sms() / L));
    a.kb_per = (a.nkb + want - 1) / want;
    a.ks = (a.nkb + a.kb_per - 1) / a.kb_per;
    a.part = part;
    a.bsum = bsum;
    a.err = net->tc->err;
    const uint32_t stage = (uint32_t)(W + KM) * 128u;
    a.nst = (int)std::min<uint32_t>(8u, (kSmemMax - 2048u) / stage);
    if (a.nst < 2) return fail(DDF_ERR_UNSUPPORTED, "weight-gradient kernel shared memory");
    a.off_bar = (uint32_t)a.nst * stage;
    const uint32_t total = a.off_bar + 256u + 1024u;
    static bool attr = false;
    if (!attr) {
        DDF_CUDA_TRY(cudaFuncSetAttribute(wgrad_all_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
        attr = true;
    }
    const int64_t items = (int64_t)L * a.ks;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<int64_t>(items, num_sms()));
    cfg.blockDim = dim3(kTThreads);
    cfg.dynamicSmemBytes = total;
    cfg.stream = s;
    cudaLaunchAttribute attrs[1];
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    DDF_CUDA_TRY(cudaLaunchKernelEx(&cfg, wgrad_all_kernel, mD, mA0, mAct, a));
    *ks_out = a.ks;
    return DDF_OK;
}

struct TcWs {
    int64_t m = 0, mp = 0;   // rows per chunk, padded to 128
    int ksplit_max = 0;
    __nv_bfloat16* act;      // a_l, l = 0..L, row-major: [mp][K0], then [mp][W] each
    uint32_t* masks;         // ReLU masks of a_1..a_{L-1}: mp x W / 32 words each; layout of their
                             // writer: [mp][W / 32] with column c at bit c (GEMM forward, read by its
                             // data-gradient GEMM), or [W / 32][mp] with the fused forward's
                             // even / odd halves (read by the chain)
    __nv_bfloat16* dl;       // deltas delta_0 .. delta_{L-1}, row-major [mp][W] each
    float* colpart;          // L x [mp / 32][W]
    float* headpart;         // [mp / 32][2W + 2]
    float* bsum;             // [L][ks][2048 / W][W] (the all-layers weight-gradient kernel)
    float* wpart;            // [ksplit][W][max(K0, W)]
    float* gx;               // [mp][K0]
    float* grad;             // [n_params]
    float* row_l1;           // [n]
    float* row_bce;          // [n]
    int* n_hit;
    double* loss_part;       // the loss reduction's partials: [256], or two per 32-row block of the
                             // chunks' padded rows (the output-layer kernel's)
    float* bpart;            // (L + 1) x kBGroups x (2W + 2)
};

int ensure_tc_ws(ddf_net_s* net, int64_t n, TcWs& ws) {
    const NetLayout& lay = net->lay;
    const int W = lay.width, L = lay.L, K0 = net->tc->K0, KM = std::max(K0, W);
    const int ntm = W / 128;   // wgrad M tiles
    ws.ksplit_max = std::max(1, num_sms() / ntm);
    // buffer sizes in bytes for chunks of mp rows, in carving order
    auto sizes = [&](size_t mp, size_t out[18]) {
        out[0] = ((size_t)K0 + (size_t)L * W) * mp * 2;                  // act (a_0 .. a_L)
        out[1] = out[2] = 0;
        out[3] = (size_t)(L - 1) * mp * W / 8 + 4;                       // masks
        out[4] = (size_t)L * mp * W * 2;                                 // dl (L arrays)
        out[5] = 0;
        out[6] = 0;
        out[7] = (size_t)L * (mp / 32) * W * 4;                          // colpart
        out[8] = (mp / 32) * (2 * W + 2) * 4;                            // headpart
        out[9] = (size_t)std::max(ws.ksplit_max, num_sms()) * W * KM * 4;  // wpart
        out[10] = mp * K0 * 4;                                           // gx
        out[11] = (size_t)lay.n_params * 4;                              // grad
        out[12] = out[13] = (size_t)n * 4;                               // row_l1, row_bce
        out[14] = 4;                                                     // n_hit
        out[15] = (size_t)std::max<int64_t>(256, 8 * ((n + 127) / 128)) * sizeof(double);   // loss partials
        out[16] = (size_t)(L + 1) * kBGroups * (2 * W + 2) * 4;          // bias-gradient partials
        out[17] = (size_t)std::max(num_sms(), L) * (2048 / W) * W * 4;   // delta column-sum partials
    };
    auto total = [&](size_t mp) {
        size_t b[18], t = 0;
        sizes(mp, b);
        for (size_t x : b) t += (x + 255) / 256 * 256;
        return t;
    };
    const size_t fixed = total(0);
    const size_t per_128 = total(128) - fixed + 18 * 256;   // bytes per 128 rows (with rounding slack)
    int64_t m = net->ws_limit > fixed ? (int64_t)((net->ws_limit - fixed) / per_128) * 128 : 0;
    m = std::max<int64_t>(128, std::min<int64_t>(m, (n + 127) / 128 * 128));
    ws.m = m;
    ws.mp = m;
    const size_t need = total((size_t)m);
    if (net->train_ws_bytes < need) {
        if (net->train_ws) cudaFree(net->train_ws);
        net->train_ws = nullptr;
        net->train_ws_bytes = 0;
        DDF_CUDA_TRY(cudaMalloc(&net->train_ws, need));
        net->train_ws_bytes = need;
    }
    size_t b[18];
    sizes((size_t)m, b);
    uint8_t* p = (uint8_t*)net->train_ws;
    void* q[18];
    for (int i = 0; i < 18; ++i) {
        q[i] = p;
        p += (b[i] + 255) / 256 * 256;
    }
    ws.act = (__nv_bfloat16*)q[0];
    ws.masks = (uint32_t*)q[3];
    ws.dl = (__nv_bfloat16*)q[4];
    ws.colpart = (float*)q[7];
    ws.headpart = (float*)q[8];
    ws.wpart = (float*)q[9];
    ws.gx = (float*)q[10];
    ws.grad = (float*)q[11];
    ws.row_l1 = (float*)q[12];
    ws.row_bce = (float*)q[13];
    ws.n_hit = (int*)q[14];
    ws.loss_part = (double*)q[15];
    ws.bpart = (float*)q[16];
    ws.bsum = (float*)q[17];
    return DDF_OK;
}

// The loss inputs of one chunk (labels) or its output cotangents.
struct ChunkTargets {
    const float* dist_gt = nullptr;
    const uint8_t* hit_gt = nullptr;
    const int* n_hit = nullptr;
    int64_t n_total = 0;
    float* row_l1 = nullptr;
    float* row_bce = nullptr;
    double* lossp = nullptr;   // per-32-row loss partials of the chunk (optional)
    bool pdl_forward = false;  // the forward may launch as a programmatic dependent of the hit count
    const float* gd = nullptr;
    const float* gl = nullptr;
};

// Encoding and forward GEMMs of rows [0, m): a_1 .. a_L row-major BF16 in ws.act (and the ReLU
// masks of a_1 .. a_{L-1} when masks is set). head (fused forward only): the output layer folded
// into the forward's last layer, a_L not stored.
int tc_forward(ddf_net_s* net, TcWs& ws, const float* o, const float* w, int64_t m, bool with_masks, cudaStream_t s,
               const TrainHeadIO* head = nullptr, bool pdl = false) {
    const NetLayout& lay = net->lay;
    TcPack* P = net->tc;
    const int W = lay.width, L = lay.L, K0 = P->K0;
    const int64_t mp = (m + 127) / 128 * 128, ld = ws.mp;
    auto act = [&](int l) { return ws.act + (l == 0 ? 0 : ((int64_t)K0 + (int64_t)(l - 1) * W) * ld); };
    auto masks = [&](int l) { return ws.masks + (int64_t)(l - 1) * ld * (W / 32); };
    int rc;
    if (K0 <= 128 && W <= 256) {
        // one persistent launch (the query's pair kernel in its training form): a_0 .. a_{L-1}
        // leave the chip by TMA stores of the A tiles, a_L and the masks from the epilogue
        CUtensorMap m0, ma;
        if ((rc = tmap(&m0, act(0), K0, K0, ld, 1, 128))) return rc;
        if ((rc = tmap(&ma, act(1), W, W, ld, L, 128))) return rc;   // L consecutive [ld][W] arrays
        return tc_train_forward(net, o, w, m, &m0, &ma, ws.masks, act(L), ld, head, pdl, s);
    }
    tenc_kernel<<<(unsigned)((mp + 127) / 128), 128, 0, s>>>(o, w, m, mp, lay.E, K0, act(0));
    DDF_LAUNCH_CHECK();

    // ---------------------------------------------------------------- forward
    for (int l = 0; l < L; ++l) {
        const int K = l == 0 ? K0 : W;
        CUtensorMap mA;
        if ((rc = tmap(&mA, act(l), K, K, m, 1, 128))) return rc;
        TArgs a{};
        a.mode = T_FWD;
        a.M = (int)m;
        a.N = W;
        a.BN = std::min(W, 256);   // width 512: two N tiles
        a.nkb = K / 64;
        a.kb_per = a.nkb;
        a.ksplit = 1;
        a.b_layer = l;
        a.bias = P->bias + (int64_t)l * W;
        a.err = P->err;
        a.out = act(l + 1);
        a.mask_out = with_masks && l + 1 < L ? masks(l + 1) : nullptr;
        if ((rc = launch_gemm(mA, P->map_fwd, a, s))) return rc;
    }
    return DDF_OK;
}

// Forward and reverse pass of rows [0, m) of one chunk; gradients accumulate into grad.
int tc_chunk(ddf_net_s* net, TcWs& ws, const float* o, const float* w, int64_t m, const ChunkTargets& tg,
             float* grad, float* gin, cudaStream_t s) {
    const NetLayout& lay = net->lay;
    TcPack* P = net->tc;
    const int W = lay.width, L = lay.L, K0 = P->K0;
    const int64_t mp = (m + 127) / 128 * 128, ld = ws.mp;
    auto act = [&](int l) { return ws.act + (l == 0 ? 0 : ((int64_t)K0 + (int64_t)(l - 1) * W) * ld); };
    auto masks = [&](int l) { return ws.masks + (int64_t)(l - 1) * ld * (W / 32); };
    auto colpart = [&](int l) { return ws.colpart + (int64_t)l * (ld / 32) * W; };
    auto dl = [&](int l) { return ws.dl + (int64_t)l * ld * W; };   // delta_l
    int rc;

    // the output layer folded into the fused forward (loss form, two-output head), or its own kernel
    const bool fold = K0 <= 128 && W <= 256 && tg.hit_gt && net->head_kind == DDF_HEAD_TWO;
    TrainHeadIO th;
    if (fold) {
        th.dist_gt = tg.dist_gt;
        th.hit_gt = tg.hit_gt;
        th.n_hit = tg.n_hit;
        th.n_total = tg.n_total;
        th.row_l1 = tg.row_l1;
        th.row_bce = tg.row_bce;
        th.lossp = tg.lossp;
        th.delta = dl(L - 1);
        th.headpart = ws.headpart;
    }
    if ((rc = tc_forward(net, ws, o, w, m, true, s, fold ? &th : nullptr, fold && tg.pdl_forward))) return rc;

    if (!fold) {   // output layer, loss and delta_{L-1}
        HeadArgs h{};
        h.aL = act(L);
        h.head = P->head;
        h.delta = dl(L - 1);
        h.colpart = colpart(L - 1);
        h.headpart = ws.headpart;
        h.m = m;
        h.mp = mp;
        h.dist_gt = tg.dist_gt;
        h.hit_gt = tg.hit_gt;
        h.n_hit = tg.n_hit;
        h.n_total = tg.n_total;
        h.row_l1 = tg.row_l1;
        h.row_bce = tg.row_bce;
        h.lossp = tg.lossp;
        h.gd_in = tg.gd;
        h.gl_in = tg.gl;
        h.head_kind = net->head_kind;
        h.head_delta = net->head_delta;
        const unsigned grid = (unsigned)((mp / 32 + 3) / 4);
        if (W == 256)
            head_kernel<256><<<grid, 128, 0, s>>>(h);
        else
            head_kernel<128><<<grid, 128, 0, s>>>(h);
        DDF_LAUNCH_CHECK();
    }

    // ---------------------------------------------------------------- reverse
    // the data-gradient chain delta_{L-2} .. delta_0 in one persistent launch where the fused
    // forward runs (and its bias-gradient column sums); otherwise one GEMM per layer below
    const bool chain = K0 <= 128 && W <= 256;
    int ks = 0;
    if (chain) {
        // then every layer's weight gradient in one launch and the split sums per layer
        if ((rc = tc_train_dgrad(net, ws.dl, m, ld, ws.masks, s))) return rc;
        if ((rc = launch_wgrad_all(net, ws.dl, act(0), act(1), m, ld, ws.wpart, ws.bsum, &ks, s))) return rc;
        const int KM = std::max(K0, W);
        DDF_CUDA_TRY(launch_k(wsum_all_kernel, dim3((unsigned)((W / 32) * (KM / 32)), (unsigned)L), dim3(32, 8), 0, s,
                              true, (const float4*)ws.wpart, ks, KM, K0, lay, grad));
    }
    for (int l = L - 1; l >= 0; --l) {
        const int K = l == 0 ? K0 : W;
        if (!chain) {   // dW_l = delta_l^T a_l, split over the rows; both operands MN-major from row-major arrays
            CUtensorMap mA, mB;
            if ((rc = tmap(&mA, dl(l), W, W, m, 1, 64))) return rc;
            if ((rc = tmap(&mB, act(l), K, K, m, 1, 64))) return rc;
            const int nkb = (int)((m + 63) / 64);
            const int want = std::max(1, std::min(ws.ksplit_max, nkb));
            const int kb_per = (nkb + want - 1) / want;
            TArgs a{};
            a.mode = T_WGRAD;
            a.mn_major = 1;
            a.M = W;
            a.N = K;
            a.BN = K;
            a.nkb = nkb;
            a.kb_per = kb_per;
            a.ksplit = (nkb + kb_per - 1) / kb_per;
            a.b_layer = 0;
            a.fout = ws.wpart;
            a.err = P->err;
            if ((rc = launch_gemm(mA, mB, a, s))) return rc;
            const int64_t tot4 = (int64_t)W * K / 4;
            wsum_kernel<<<(unsigned)((tot4 + 31) / 32), dim3(32, 8), 0, s>>>((const float4*)ws.wpart, a.ksplit, W, K,
                                                                            l == 0 ? lay.E : W, l == 0,
                                                                            grad + lay.w_off[l]);
            DDF_LAUNCH_CHECK();
        }
        if (l > 0 && !chain) {   // delta_{l-1} = (delta_l W_l) * 1[a_l > 0]
            CUtensorMap mA;
            if ((rc = tmap(&mA, dl(l), W, W, m, 1, 128))) return rc;
            TArgs a{};
            a.mode = T_DGRAD;
            a.M = (int)m;
            a.N = W;
            a.BN = W;
            a.nkb = W / 64;
            a.kb_per = a.nkb;
            a.ksplit = 1;
            a.b_layer = l;
            a.mask_in = masks(l);
            a.out = dl(l - 1);
            a.colpart = colpart(l - 1);
            a.err = P->err;
            if ((rc = launch_gemm(mA, P->map_bwd, a, s))) return rc;
        } else if (l == 0 && gin) {   // d/d(internal inputs) = delta_0 W_0, then the encoding's Jacobian
            CUtensorMap mA, mB;
            if ((rc = tmap(&mA, dl(0), W, W, m, 1, 128))) return rc;
            if ((rc = tmap(&mB, P->w_bwd, W, W, W, L, K0))) return rc;
            TArgs a{};
            a.mode = T_STORE;
            a.M = (int)m;
            a.N = K0;
            a.BN = K0;
            a.nkb = W / 64;
            a.kb_per = a.nkb;
            a.ksplit = 1;
            a.b_layer = 0;
            a.fout = ws.gx;
            a.err = P->err;
            if ((rc = launch_gemm(mA, mB, a, s))) return rc;
            tenc_backward_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(o, w, m, lay.E, K0, ws.gx, gin);
            DDF_LAUNCH_CHECK();
        }
    }
    // bias gradients: from the weight-gradient kernel's column sums on the chain path, from the
    // per-32-row column sums of the head and the data-gradient GEMMs otherwise
    const unsigned gx = (unsigned)((2 * W + 2 + 31) / 32);
    const int64_t lrows = chain ? (int64_t)ks * (2048 / W) : mp / 32;
    DDF_CUDA_TRY(launch_k(bgrad_partial_kernel, dim3(gx, (unsigned)(L + 1), kBGroups), dim3(32, 8), 0, s, true,
                          (const float*)(chain ? ws.bsum : ws.colpart), lrows, chain ? lrows * W : (ld / 32) * W,
                          (const float*)ws.headpart, (int64_t)(mp / 32), lay, ws.bpart));
    DDF_CUDA_TRY(launch_k(bgrad_final_kernel, dim3(gx, (unsigned)(L + 1)), dim3(32), 0, s, true, (const float*)ws.bpart,
                          lay, grad));
    return DDF_OK;
}

// Calibration rays for the FP8 activation scales: origins uniform in the unit ball, directions
// uniform on the sphere, from Philox4x32-10 (key = seed, counter = (ray, 0, slot, 0)).
__global__ void cal_rays_kernel(float* __restrict__ o, float* __restrict__ w, int n, uint64_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    const uint4 a = philox4x32_10(make_uint4((uint32_t)i, 0u, 0u, 0u), key);
    const uint4 b = philox4x32_10(make_uint4((uint32_t)i, 0u, 1u, 0u), key);
    const float z0 = 1.f - 2.f * u24(a.x), p0 = 6.2831853f * u24(a.y), r0 = cbrtf(u24(a.z));
    const float s0 = sqrtf(fmaxf(0.f, 1.f - z0 * z0));
    o[3 * i + 0] = r0 * s0 * cosf(p0);
    o[3 * i + 1] = r0 * s0 * sinf(p0);
    o[3 * i + 2] = r0 * z0;
    const float z1 = 1.f - 2.f * u24(b.x), p1 = 6.2831853f * u24(b.y);
    const float s1 = sqrtf(fmaxf(0.f, 1.f - z1 * z1));
    w[3 * i + 0] = s1 * cosf(p1);
    w[3 * i + 1] = s1 * sinf(p1);
    w[3 * i + 2] = z1;
}

// amax[c] = max over rows of |a[r][c]| (BF16 [m][W]); block (32, 8): 32 columns x 8 row lanes.
__global__ void colmax_kernel(const __nv_bfloat16* __restrict__ a, int64_t m, int W, float* __restrict__ amax) {
    const int c = blockIdx.x * 32 + threadIdx.x;
    __shared__ float red[8][33];
    float mx = 0.f;
    if (c < W)
        for (int64_t r = threadIdx.y; r < m; r += 8) mx = fmaxf(mx, fabsf(__bfloat162float(a[r * W + c])));
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0 && c < W) {
        for (int k = 1; k < 8; ++k) mx = fmaxf(mx, red[k][threadIdx.x]);
        amax[c] = mx;
    }
}

constexpr int kCalRows = 8192;
constexpr uint64_t kCalSeed = 0x43414C4942ull;

}  // namespace

bool tct_supported(const ddf_net_s* net) {
    if (net->is_sphere || !net->tc) return false;
    if (net->precision != DDF_BF16 && net->precision != DDF_FP8) return false;
    const int W = net->lay.width;
    return (W == 128 || W == 256) && net->tc->K0 <= 256;
}

int tct_train_step(ddf_net_s* net, const float* o, const float* w, const float* dist_gt, const uint8_t* hit_gt,
                   int64_t n, const ddf_adam* opt, float* loss, cudaStream_t s) {
    TcWs ws;
    int rc = ensure_tc_ws(net, n, ws);
    if (rc) return rc;
    DDF_CUDA_TRY(cudaMemsetAsync(ws.grad, 0, sizeof(float) * net->lay.n_params, s));
    if ((rc = count_hits(hit_gt, n, ws.n_hit, s))) return rc;
    // BF16 handles with the plain two-output head: the output-layer kernel leaves per-32-row loss
    // partials and one launch takes the loss, the Adam step and the repacking
    const bool fused_tail = net->precision == DDF_BF16 && !net->wn_p && !head_single(net);
    for (int64_t r0 = 0; r0 < n; r0 += ws.m) {
        const int64_t m = std::min(ws.m, n - r0);
        ChunkTargets tg;
        tg.dist_gt = dist_gt + r0;
        tg.hit_gt = hit_gt + r0;
        tg.n_hit = ws.n_hit;
        tg.n_total = n;
        tg.row_l1 = ws.row_l1 + r0;
        tg.row_bce = ws.row_bce + r0;
        tg.lossp = fused_tail ? ws.loss_part + 2 * (r0 / 32) : nullptr;
        tg.pdl_forward = r0 == 0;   // later chunks' forwards overwrite what the previous chunk reads
        if ((rc = tc_chunk(net, ws, o + 3 * r0, w + 3 * r0, m, tg, ws.grad, nullptr, s))) return rc;
    }
    if (fused_tail) {
        float c1, c2;
        if ((rc = adam_prepare(net, opt, &c1, &c2, s))) return rc;
        net->master_t_stale = true;   // the FP32 transposed copy is rebuilt by the next FP32 query
        return tc_adam_pack(net, ws.grad, opt, c1, c2, ws.loss_part, (n + 127) / 128 * 4, ws.n_hit, n, loss, s);
    }
    if (loss && (rc = loss_reduce(ws.row_l1, ws.row_bce, n, ws.n_hit, loss, ws.loss_part, s))) return rc;
    return adam_and_repack(net, ws.grad, opt, s);
}

int tct_backward(ddf_net_s* net, const float* o, const float* w, int64_t n, const float* gdist,
                 const float* glogit, float* gweights, float* ginput, cudaStream_t s) {
    TcWs ws;
    int rc = ensure_tc_ws(net, n, ws);
    if (rc) return rc;
    DDF_CUDA_TRY(cudaMemsetAsync(gweights, 0, sizeof(float) * net->lay.n_params, s));
    for (int64_t r0 = 0; r0 < n; r0 += ws.m) {
        const int64_t m = std::min(ws.m, n - r0);
        ChunkTargets tg;
        tg.gd = gdist ? gdist + r0 : nullptr;
        tg.gl = glogit ? glogit + r0 : nullptr;
        if ((rc = tc_chunk(net, ws, o + 3 * r0, w + 3 * r0, m, tg, gweights, ginput ? ginput + 6 * r0 : nullptr,
                           s)))
            return rc;
    }
    return DDF_OK;
}

int tct_calibrate_fp8(ddf_net_s* net, float* d_amax, cudaStream_t s) {
    const NetLayout& lay = net->lay;
    const int W = lay.width, L = lay.L;
    TcWs ws;
    int rc = ensure_tc_ws(net, kCalRows, ws);
    if (rc) return rc;
    float* o = ws.gx;                      // scratch for the calibration rays
    float* w = ws.gx + 3 * kCalRows;
    cal_rays_kernel<<<(kCalRows + 255) / 256, 256, 0, s>>>(o, w, kCalRows, kCalSeed);
    DDF_LAUNCH_CHECK();
    if ((rc = tc_forward(net, ws, o, w, kCalRows, false, s))) return rc;
    DDF_CUDA_TRY(cudaMemsetAsync(d_amax, 0, sizeof(float) * W, s));   // layer 0: fixed scale
    const int64_t ld = ws.mp;
    for (int l = 1; l < L; ++l) {
        const __nv_bfloat16* a = ws.act + ((int64_t)net->tc->K0 + (int64_t)(l - 1) * W) * ld;
        colmax_kernel<<<(W + 31) / 32, dim3(32, 8), 0, s>>>(a, kCalRows, W, d_amax + (int64_t)l * W);
        DDF_LAUNCH_CHECK();
    }
    return DDF_OK;
}

}  // namespace ddf

