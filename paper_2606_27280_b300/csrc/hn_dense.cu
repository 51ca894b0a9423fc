// Dense prefix scan on the 5th-generation tensor cores (tcgen05), Phase 1 and
// Phase 2 of Algorithm 1 (§3.3) for a BF16 major prefix.
//
// For a tile of 128 queries (A, K-major) and 256 database entries (B,
// K-major) one tcgen05.mma per 16 prefix columns computes the 128 x 256 block
// of prefix scores s~ = q^ . x^ with FP32 accumulation into tensor memory.
// Products of two BF16 values are exact in FP32; the sum carries at most the
// accumulation error bounded in the Phase-2 slack (hn_prep.cu).
//
// Phase 1 only looks for good threshold candidates (their full scores are
// certified later), so it runs on an FP16 copy of the prefix with FP16
// accumulation and reduces packed f16 pairs; Phase 2, the certified bound test,
// runs on the BF16 prefix with FP32 accumulation.
//
// Persistent CTAs (one per SM, 10 warps):
//   warp 0   producer: 1-D bulk copies of the query tile (once per work unit)
//            and of each 8 KB entry tile into a ring of shared-memory stages;
//   warp 1   allocates 512 TMEM columns; one lane issues the MMAs into one of
//            two 256-column accumulators and commits them to mbarriers;
//   warps 2-17 epilogue (4 per SM sub-partition): TMEM -> registers (thread =
//            query row, 64 accumulator columns per warp), one max tree, then
//              Phase 1: running best score and its 64-entry segment per (query, chunk, segment);
//              Phase 2: entries with s~ >= tau_q appended to q's survivor slots.
// A work unit is (query tile, contiguous chunk of entry tiles); units are
// numbered chunk-major so that the CTAs running together read the same entry
// tiles, which then come from L2.
// Every mbarrier wait gives up after 2 s of global time: the CTA raises a
// shared abort flag, the others leave their loops, copies and MMAs in flight
// are drained (again with a limit), TMEM is released and the status word
// ST_TIMEOUT tells the host.
#include "hn_internal.cuh"
#include "hn_sm100.cuh"

namespace hn {
using namespace sm100;

constexpr int kEpiWarps = 16;  // 4 per SM sub-partition, 64 accumulator columns each
constexpr int kDenseThreads = (2 + kEpiWarps) * 32;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr int kMinDenseSmem = 120 * 1024;  // forces one CTA (and one TMEM owner) per SM

struct DenseParams {
    const void *pre;              // entries, UMMA core-matrix order, n_tiles * 256 rows (FP16 or BF16)
    const void *qpre;             // queries, same order, n_qt * 128 rows
    int64_t n, n_tiles, nq;
    int64_t n_qt, tiles_per_chunk, n_units;
    const float *tau;
    unsigned long long *cand;     // [nq][4 * chunks] Phase-1 (best score, segment id) per (query, chunk, column segment)
    int32_t *bucket, *count;
    int32_t cap;
    int32_t *status;
};

constexpr int kLcap = 32;  // Phase-2 survivors staged per epilogue thread before a flush

template <int KP>
struct DenseCfg {
    static constexpr uint32_t kB = kTileE * KP * 2;  // bytes of one entry tile
    static constexpr uint32_t kA = kTileQ * KP * 2;  // bytes of one query tile
    static constexpr int kStages = (64 * 1024) / kB < 2 ? 2 : (64 * 1024) / kB;
    static constexpr uint32_t kSurvOff = kStages * kB + 2 * kA;
    static constexpr uint32_t kBarOff = kSurvOff + kLcap * kEpiWarps * 32 * 4;  // [kLcap][512] entry ids
    static constexpr int kBars = 2 * kStages + 9;
    static constexpr uint32_t kSmem = kBarOff + kBars * 8 + 16;
};

// Max of 16 consecutive scores, pairwise (15 two-input max, depth 4).
__device__ __forceinline__ float max16(const float *v) {
    float a[8], b[4];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fmaxf(v[2 * i], v[2 * i + 1]);
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = fmaxf(a[2 * i], a[2 * i + 1]);
    return fmaxf(fmaxf(b[0], b[1]), fmaxf(b[2], b[3]));
}

// Max of 64 f16 scores held as 32 packed pairs (31 packed max + 1), as a float.
__device__ __forceinline__ float max64_f16(uint32_t (&r)[32]) {
    __half2 h[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) h[i] = *reinterpret_cast<__half2 *>(&r[i]);
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
        for (int i = 0; i < w; ++i) h[i] = __hmax2(h[2 * i], h[2 * i + 1]);
    return fmaxf(__low2float(h[0]), __high2float(h[0]));
}

template <int KP, int PHASE>
__global__ void __launch_bounds__(kDenseThreads, 1) k_dense_scan(const DenseParams p) {
    using C = DenseCfg<KP>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;
    uint8_t *sA = smem + C::kStages * C::kB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::kBarOff);
    uint64_t *b_full = bars, *b_empty = bars + C::kStages;
    uint64_t *a_full = bars + 2 * C::kStages, *a_empty = a_full + 2;
    uint64_t *acc_full = a_empty + 2, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::kStages; ++i) {
            mbar_init(smem_u32(&b_full[i]), 1);
            mbar_init(smem_u32(&b_empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&a_full[i]), 1);
            mbar_init(smem_u32(&a_empty[i]), 1);
            mbar_init(smem_u32(&acc_full[i]), 1);
            mbar_init(smem_u32(&acc_empty[i]), kEpiWarps);  // one elected arrive per epilogue warp
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_u32(tmem_slot), 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t G = gridDim.x;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t stage = 0, sphase = 0, abuf = 0, aphase = 0;
            uint32_t issued = 0;               // stages / A buffers that received a copy
            uint32_t last_par = 0;             // parity of the last copy per stage / A buffer
            bool ok = true;
            for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
                const int64_t qt = u % p.n_qt, ch = u / p.n_qt;
                const int64_t t0 = ch * p.tiles_per_chunk, t1 = min64(p.n_tiles, t0 + p.tiles_per_chunk);
                if (!(ok = mbar_wait(smem_u32(&a_empty[abuf]), aphase ^ 1, abort_flag, kWaitLimitNs))) break;
                mbar_arrive_expect_tx(smem_u32(&a_full[abuf]), C::kA);
                bulk_g2s(smem_u32(sA + abuf * C::kA), static_cast<const char *>(p.qpre) + qt * C::kA, C::kA,
                         smem_u32(&a_full[abuf]));
                issued |= 1u << (24 + abuf);
                last_par = (last_par & ~(1u << (24 + abuf))) | (aphase << (24 + abuf));
                if (++abuf == 2) { abuf = 0; aphase ^= 1; }
                for (int64_t t = t0; t < t1; ++t) {
                    if (!(ok = mbar_wait(smem_u32(&b_empty[stage]), sphase ^ 1, abort_flag, kWaitLimitNs))) break;
                    mbar_arrive_expect_tx(smem_u32(&b_full[stage]), C::kB);
                    bulk_g2s(smem_u32(sB + stage * C::kB), static_cast<const char *>(p.pre) + t * C::kB, C::kB,
                             smem_u32(&b_full[stage]));
                    issued |= 1u << stage;
                    last_par = (last_par & ~(1u << stage)) | (sphase << stage);
                    if (++stage == C::kStages) { stage = 0; sphase ^= 1; }
                }
            }
            // copies still in flight must land before this CTA's shared memory goes away
            for (int s = 0; s < C::kStages; ++s)
                if (issued & (1u << s)) mbar_drain(smem_u32(&b_full[s]), (last_par >> s) & 1, kWaitLimitNs);
            for (int s = 0; s < 2; ++s)
                if (issued & (1u << (24 + s))) mbar_drain(smem_u32(&a_full[s]), (last_par >> (24 + s)) & 1, kWaitLimitNs);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            // Phase 1: FP16 operands, FP16 accumulator; Phase 2: BF16 operands, FP32 accumulator
            constexpr uint32_t idesc = PHASE == 1 ? idesc_f16_f16(kTileQ, kTileE) : idesc_bf16_f32(kTileQ, kTileE);
            uint32_t stage = 0, sphase = 0, abuf = 0, aphase = 0, acc = 0, accphase = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
                const int64_t ch = u / p.n_qt;
                const int64_t t0 = ch * p.tiles_per_chunk, t1 = min64(p.n_tiles, t0 + p.tiles_per_chunk);
                if (!(ok = mbar_wait(smem_u32(&a_full[abuf]), aphase, abort_flag, kWaitLimitNs))) break;
                tc_fence_after();
                const uint32_t a_addr = smem_u32(sA + abuf * C::kA);
                for (int64_t t = t0; t < t1; ++t) {
                    if (!(ok = mbar_wait(smem_u32(&acc_empty[acc]), accphase ^ 1, abort_flag, kWaitLimitNs))) break;
                    if (!(ok = mbar_wait(smem_u32(&b_full[stage]), sphase, abort_flag, kWaitLimitNs))) break;
                    tc_fence_after();
                    const uint32_t b_addr = smem_u32(sB + stage * C::kB);
#pragma unroll
                    for (int kk = 0; kk < KP / 16; ++kk) {
                        // 16 columns = two core matrices along K, 128 B apart; 8-row groups KP*16 B apart
                        const uint64_t ad = smem_desc(a_addr + kk * 256, 128, KP * 16);
                        const uint64_t bd = smem_desc(b_addr + kk * 256, 128, KP * 16);
                        umma_bf16(tmem + acc * kTileE, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    umma_commit(smem_u32(&b_empty[stage]));
                    umma_commit(smem_u32(&acc_full[acc]));
                    if (++stage == C::kStages) { stage = 0; sphase ^= 1; }
                    if (++acc == 2) { acc = 0; accphase ^= 1; }
                }
                umma_commit(smem_u32(&a_empty[abuf]));
                if (++abuf == 2) { abuf = 0; aphase ^= 1; }
            }
            // every MMA issued so far must finish before TMEM is released
            umma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0, kWaitLimitNs);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;          // TMEM lanes this warp may read: 32*quarter ..
        const int seg = (warp - 2) >> 2;       // accumulator columns 64*seg .. 64*seg + 63
        const int row = quarter * 32 + lane;
        const int et = threadIdx.x - 64;       // epilogue thread 0..511
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        uint32_t *sbuf = reinterpret_cast<uint32_t *>(smem + C::kSurvOff);  // [kLcap][512]
        uint32_t acc = 0, accphase = 0;
        bool ok = true;
        for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
            const int64_t qt = u % p.n_qt, ch = u / p.n_qt;
            const int64_t t0 = ch * p.tiles_per_chunk, t1 = min64(p.n_tiles, t0 + p.tiles_per_chunk);
            const int64_t q = qt * kTileQ + row;
            const bool qvalid = q < p.nq;
            const float thr = (PHASE == 2 && qvalid) ? p.tau[q] : INFINITY;
            float best = -INFINITY;
            int32_t bseg = -1;
            int lc = 0;
            // Phase 2: move this thread's staged survivors to its query's slots
            auto flush = [&]() {
                const int slot = atomicAdd(p.count + q, lc);
                for (int j = 0; j < lc; ++j)
                    if (slot + j < p.cap) p.bucket[q * p.cap + slot + j] = (int32_t)sbuf[j * 512 + et];
                lc = 0;
            };
            // entry ids fit in 32 bits (n < 2^31 - 256 is enforced by hn_index_build)
            const int32_t n32 = (int32_t)p.n;
            for (int32_t t = (int32_t)t0; t < (int32_t)t1; ++t) {
                if (!(ok = mbar_wait(smem_u32(&acc_full[acc]), accphase, abort_flag, kWaitLimitNs))) break;
                tc_fence_after();
                const int32_t e0 = t * kTileE + seg * 64;
                if (PHASE == 1) {
                    uint32_t r[32];
                    tmem_ld64_f16(tmem + acc * kTileE + seg * 64 + lane_addr, r);
                    // the scores are in registers: hand the accumulator back to the MMA warp now
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
                    if (++acc == 2) { acc = 0; accphase ^= 1; }
                    // running best score and the 64-entry segment holding it; the entry
                    // itself is recovered by the threshold kernel
                    const float m = max64_f16(r);
                    if (m > best && e0 < n32) { best = m; bseg = t * 4 + seg; }
                } else {
                    float v[64];
                    tmem_ld64(tmem + acc * kTileE + seg * 64 + lane_addr, v);
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_u32(&acc_empty[acc]));
                    if (++acc == 2) { acc = 0; accphase ^= 1; }
                    float g[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) g[k] = max16(v + 16 * k);
                    const float m = fmaxf(fmaxf(g[0], g[1]), fmaxf(g[2], g[3]));
                    if (m >= thr) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (g[k] >= thr) {
                                uint32_t mask = 0;
#pragma unroll
                                for (int i = 0; i < 16; ++i) mask |= (v[16 * k + i] >= thr ? 1u : 0u) << i;
                                const int32_t ek = e0 + 16 * k;
                                if (ek + 16 > n32) mask &= ek >= n32 ? 0u : ((1u << (uint32_t)(n32 - ek)) - 1u);
                                if (lc + __popc(mask) > kLcap) flush();
                                while (mask) {
                                    const int i = __ffs(mask) - 1;
                                    mask &= mask - 1;
                                    sbuf[lc * 512 + et] = (uint32_t)(ek + i);
                                    ++lc;
                                }
                            }
                        }
                    }
                }
            }
            // one writer per (query, chunk, segment): no atomics, every slot written
            if (PHASE == 1 && qvalid)
                p.cand[q * (4 * (p.n_units / p.n_qt)) + 4 * ch + seg] =
                    bseg >= 0 ? pack_best(best, (uint32_t)bseg) : 0ull;
            if (PHASE == 2 && lc > 0) flush();
        }
    }

    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status + ST_TIMEOUT, 1);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

static int g_num_sms = 0;

static int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 148;
    }
    return g_num_sms;
}

// About 32 work units per CTA, numbered chunk-major so that the running CTAs
// share entry tiles in L2.
static void dense_chunking(int64_t n_tiles, int64_t n_qt, int G, int64_t *tiles_per_chunk, int64_t *chunks) {
    int64_t c = (32ll * G + n_qt - 1) / n_qt;
    c = max64(1, min64(c, n_tiles));
    const int64_t tpc = (n_tiles + c - 1) / c;
    *tiles_per_chunk = tpc;
    *chunks = (n_tiles + tpc - 1) / tpc;
}

int64_t dense_cand_slots(const Index &ix, int64_t nq) {
    int64_t tpc = 0, chunks = 0;
    dense_chunking(ix.n_tiles, (nq + kTileQ - 1) / kTileQ, num_sms(), &tpc, &chunks);
    return 4 * chunks;
}

bool dense_scan_supported(const Index &ix) {
    return ix.prefix == HN_PREFIX_BF16 && (ix.k_pad16 == 16 || ix.k_pad16 == 32 || ix.k_pad16 == 64);
}

template <int KP, int PHASE>
static cudaError_t launch_kp(const DenseParams &p, int grid, cudaStream_t st) {
    using C = DenseCfg<KP>;
    const int smem = (int)C::kSmem < kMinDenseSmem ? kMinDenseSmem : (int)C::kSmem;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_dense_scan<KP, PHASE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_dense_scan<KP, PHASE><<<grid, kDenseThreads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_dense_scan(const Index &ix, int64_t nq, int phase, cudaStream_t st) {
    if (!dense_scan_supported(ix)) return cudaErrorNotSupported;
    const Workspace &ws = ix.ws;
    DenseParams p{};
    p.pre = phase == 1 ? (const void *)ix.pre16h : (const void *)ix.pre16;
    p.qpre = phase == 1 ? (const void *)ws.qpre16h : (const void *)ws.qpre16;
    p.n = ix.n;
    p.n_tiles = ix.n_tiles;
    p.nq = nq;
    p.n_qt = (nq + kTileQ - 1) / kTileQ;
    const int G = num_sms();
    int64_t chunks = 0;
    dense_chunking(ix.n_tiles, p.n_qt, G, &p.tiles_per_chunk, &chunks);
    p.n_units = p.n_qt * chunks;
    p.tau = ws.tau;
    p.cand = ws.cand;
    p.bucket = ws.bucket;
    p.count = ws.count;
    p.cap = ws.bucket_cap;
    p.status = ws.status;
    const int grid = (int)min64(G, p.n_units);
    switch (ix.k_pad16) {
        case 16: return phase == 1 ? launch_kp<16, 1>(p, grid, st) : launch_kp<16, 2>(p, grid, st);
        case 32: return phase == 1 ? launch_kp<32, 1>(p, grid, st) : launch_kp<32, 2>(p, grid, st);
        case 64: return phase == 1 ? launch_kp<64, 1>(p, grid, st) : launch_kp<64, 2>(p, grid, st);
    }
    return cudaErrorNotSupported;
}

}  // namespace hn
