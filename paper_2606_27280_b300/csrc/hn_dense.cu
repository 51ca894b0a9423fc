// Dense prefix scan on the 5th-generation tensor cores (tcgen05), Phase 1 and
// Phase 2 of Algorithm 1 (§3.3) for a BF16 (or FP8) major prefix.
//
// The one-pass form (PHASE 4) computes the prefix product once: its epilogue keeps, per
// (query, 32-entry group), an 8-bit code of the group's largest score (hn_internal.cuh)
// and, per (query, chunk, tile parity), the best group as a threshold candidate.  The
// threshold kernel then scores the candidates in full and k_dense_extract_codes takes the
// survivors from the groups whose code reaches code(tau_q).  The codes cost one byte per 32
// scores of HBM traffic (written once, read once), against a second tensor-core pass over
// all Q x N scores.  The two-pass form runs Algorithm 1's phases as two scans: Phase 1 is
// the PHASE-4 kernel without its code map (threshold candidates only), then PHASE 2 marks,
// against the threshold, one bit per 32-entry group whose maximum reaches tau_q, and
// k_dense_extract scores the flagged groups.  PHASE 3 writes every FP32 score to memory
// (verification only).
//
// A work unit pairs 256 queries (two 128-row A tiles, K-major) with a stream of 128-entry
// B tiles (K-major).  BF16 PHASE 4 with two or more tiles a ring stage: one N = 256 MMA per
// 16 prefix columns computes a 128-query half against a pair of tiles; otherwise two N = 128
// MMAs per tile, one per query half.  Reusing every B tile for 256 queries halves the L2 ->
// shared-memory traffic of 128-query tiles, which measured as the limiting stream.  Products
// of two BF16 values are exact in FP32; the sum carries at most the accumulation error
// bounded in the slack of the bound test (hn_prep.cu).
//
// FP8 index (F8): kind::f8f6f4 with e4m3 operands.  An entry tile holds kp e4m3 bytes per
// entry plus its per-entry scales and error terms.  Each MMA takes K = 32 bytes: the query
// side supplies 16 hi and 16 lo bytes of one 16-column group, the entry side the same 16
// bytes twice (its K-direction core-matrix stride is 0), so acc = (hi + lo) . x^ costs no
// extra entry bytes.  The epilogue applies the per-entry scale and error term, u = fma(acc,
// s_i / 256, b_i) (PHASE 2 and 3), or bounds a group's scores from its largest raw
// accumulator (PHASE 4); it reads these from the stage, so every epilogue warp releases
// the stage.
//
// Persistent CTAs (one per SM, 20 warps):
//   warp 0   producer: 1-D bulk copies of the 256-query unit (once per work unit) and of
//            16 KB stages of entry tiles into a ring in shared memory;
//   warps 1-2 allocate 512 TMEM columns (warp 1); one lane each issues the MMAs into its
//            own 256-column accumulator and commits them;
//   warp 3   idle (completes the first warp group for the register split);
//   warps 4-19 epilogue (4 per SM sub-partition), TMEM -> registers with thread = query row.
// A work unit is (query tile, contiguous chunk of entry tiles); units are numbered
// chunk-major so that the CTAs running together read the same entry tiles, which then
// come from L2.
// Every mbarrier wait gives up after 2 s of global time: the CTA raises a shared abort
// flag, the others leave their loops, copies and MMAs in flight are drained (again with a
// limit), TMEM is released and the status word ST_TIMEOUT tells the host.
#include <algorithm>

#include <cuda_fp8.h>

#include "hn_internal.cuh"
#include "hn_sm100.cuh"

namespace hn {
using namespace sm100;

constexpr int kIssuers = 2;                      // MMA-issuing threads, one per accumulator buffer
constexpr int kEpiWarps = 16;                    // 4 per SM sub-partition, 64 accumulator columns each
// warp 0 producer, warps 1..kIssuers MMA issuers, warp 3 idle (it completes the first warpgroup,
// so that warps 4.. form whole warpgroups for setmaxnreg), warps 4..19 epilogue
constexpr int kEpiWarp0 = 4;
constexpr int kDenseThreads = (kEpiWarp0 + kEpiWarps) * 32;
// Register split of the one-pass form with setmaxnreg (REG): 640 threads launched at 96 registers
// = 61,440; the first warpgroup (producer, issuers, idle) drops to 56, the four epilogue
// warpgroups rise to 104: 128 * 56 + 512 * 104 = 60,416.  The host launches that form only when the
// kernel's register count is exactly kRegLaunch (otherwise an increase could wait forever).
constexpr int kRegLaunch = 96, kRegLow = 56, kRegHigh = 104;
static_assert(128 * kRegLow + 512 * kRegHigh <= kDenseThreads * kRegLaunch, "setmaxnreg split above the launch budget");
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // default main-loop wait limit, and every drain's
constexpr int kMinDenseSmem = 120 * 1024;  // forces one CTA (and one TMEM owner) per SM

// One index and query batch of a dense launch.  A launch has one group, or (the one-pass
// form of batched serving) several that share the tile format, with their work units
// numbered group by group.
struct DenseGroup {
    const void *pre;              // entries, UMMA core-matrix order, n_tiles * 128 rows (BF16 or FP8 tiles)
    const void *qpre;             // queries, same order, n_qt * 256 rows
    int64_t n, n_tiles, nq;
    int64_t n_qt, tiles_per_chunk, chunks;
    int64_t unit0;                // global number of the group's first work unit
    const float *tau;
    unsigned long long *cand;     // [nq][2 * chunks] PHASE 4: (best group score, 32-entry group id)
                                  //   per (query, chunk, tile parity)
    uint32_t *gbits;              // group map: PHASE 2 [chunk][half][word][n_qt * 256] passing-group bits,
                                  //   16 tiles a word; PHASE 4 [chunk][tile][n_qt * 256] the 4 group codes
                                  //   of a tile in a word
    int64_t words;                // PHASE 2: words per (chunk, half), ceil(tiles_per_chunk / 16);
                                  //   PHASE 4: words per chunk, tiles_per_chunk
    float code_inv;               // PHASE 4: the group code (hn_internal.cuh)
};

struct DenseParams {
    DenseGroup g;                 // the group of a single-group launch (n_groups == 0)
    const DenseGroup *groups;     // n_groups > 0: the groups' descriptors (device memory)
    int32_t n_groups;
    int64_t n_units;              // work units of all groups
    float code_base;              // PHASE 4: the group code
    float *dump;                  // PHASE 3: [nq][n] every FP32 score (Phase-2 arithmetic)
    uint64_t wait_ns;             // limit of every main-loop wait (the drains keep kWaitLimitNs)
    int32_t *status;
    int32_t stall;                // failure-path test: the producer stops after each CTA's first unit
    int32_t plain;                // one-pass form: launch the unsplit instantiation (test hook)
};
constexpr int kDQ = 256;   // queries per work unit (two MMA A tiles)
constexpr int kDE = 128;   // entries per B tile (MMA N)

// Group of work unit u in a multi-group launch (the last group whose unit0 <= u).
__device__ __forceinline__ const DenseGroup &group_of(const DenseParams &p, int64_t u) {
    int lo = 0, hi = p.n_groups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.groups[mid].unit0 <= u) lo = mid; else hi = mid - 1;
    }
    return p.groups[lo];
}

// Measured on B300: one thread issues a 1-D bulk copy every ~350 cycles whatever
// its size, and a tcgen05.commit costs ~220 cycles.  So a ring stage holds
// several B tiles filled by one 16 KB copy, stages are released by the epilogue
// with plain mbarrier arrivals (no commit), and two threads issue the MMAs, one
// per accumulator buffer, each committing once per tile of its own.
template <int KP, int PHASE, bool F8>
struct DenseCfg {
    static constexpr uint32_t kB = F8 ? (uint32_t)kF8TileBytes(KP) : kDE * KP * 2;  // bytes of one entry tile
    static constexpr int kTPS = kB >= 16384 ? 1 : 16384 / kB;       // entry tiles per stage
    static constexpr uint32_t kStageBytes = kTPS * kB;
    static constexpr uint32_t kA = kDQ * KP * 2;                    // bytes of one query unit (FP8: hi + lo)
    static constexpr uint32_t kSurvBytes = 0;
    // ring: 160 KB, capped by what the 227 KB of shared memory leaves after the two
    // query units and the barriers
    static constexpr uint32_t kRoom = 225 * 1024 - 2 * kA - kSurvBytes;
    static constexpr uint32_t kWant = 160 * 1024;
    static constexpr uint32_t kRing = kWant < kRoom ? kWant : kRoom;
    static constexpr int kStages = kRing / kStageBytes < 2 ? 2 : kRing / kStageBytes;
    static constexpr uint32_t kSurvOff = kStages * kStageBytes + 2 * kA;
    static constexpr uint32_t kBarOff = kSurvOff + kSurvBytes;
    // b_full[S], b_empty[S], a_full[2], a_empty[2], acc_full[2], acc_empty[2], drain[kIssuers]
    static constexpr int kBars = 2 * kStages + 8 + kIssuers;
    static constexpr uint32_t kSmem = kBarOff + kBars * 8 + 16;
    static_assert(kSmem <= 232448, "dense scan shared memory above the 227 KB limit");
};

// Max of 16 consecutive scores: seven three-input max and one two-input max.
// Measured on B300, the two- and three-input f32 max both issue at half rate
// (about 1.9 warp instructions per clock per SM), so the three-input form does two
// reductions for the cost of one.
__device__ __forceinline__ float max16(const float *v) {
    const float a0 = fmax3(v[0], v[1], v[2]), a1 = fmax3(v[3], v[4], v[5]), a2 = fmax3(v[6], v[7], v[8]);
    const float a3 = fmax3(v[9], v[10], v[11]), a4 = fmax3(v[12], v[13], v[14]);
    return fmaxf(fmax3(a0, a1, a2), fmax3(a3, a4, v[15]));
}

// Max of 32 consecutive scores: fifteen three-input max and one two-input max (the
// 31 reductions in 16 half-rate instructions).
__device__ __forceinline__ float max32(const float *v) {
    float a[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) a[i] = fmax3(v[3 * i], v[3 * i + 1], v[3 * i + 2]);
    const float b0 = fmax3(a[0], a[1], a[2]), b1 = fmax3(a[3], a[4], a[5]), b2 = fmax3(a[6], a[7], a[8]);
    const float b3 = fmax3(a[9], v[30], v[31]);
    return fmaxf(fmax3(b0, b1, b2), b3);
}

// 2^23 + code(g) as binary32 bits before the upper clamp of code_group_bits: byte 0 is
// the code while RU(g inv + 2^23 + 128) stays below 2^23 + 256.
__device__ __forceinline__ uint32_t code_bits_unclamped(float g, float inv, float base) {
    return __float_as_uint(__fmaf_ru(g, inv, base));
}

// MULTI: the launch covers several groups (p.groups); otherwise the one group p.g, read in
// place from the kernel parameters.
// REG (one-pass form only, single or multi-group): the setmaxnreg register split, and two
// reducing TMEM loads in flight per epilogue warp instead of one.
template <int KP, int PHASE, bool F8, bool MULTI = false, bool REG = false>
__global__ void __launch_bounds__(kDenseThreads, 1) k_dense_scan(const __grid_constant__ DenseParams p) {
    // PHASE 4: the one-pass form; PHASE 1: its epilogue without the code map (the two-pass
    // form's Phase 1, threshold candidates only)
    constexpr bool ONEPASS = PHASE == 4 || PHASE == 1;
    constexpr bool CODES = PHASE == 4;
    static_assert(!REG || ONEPASS, "the register split serves the one-pass epilogue");
    using C = DenseCfg<KP, PHASE, F8>;
    // PAIR (one-pass BF16, at least two entry tiles a ring stage): an accumulator buffer holds
    // one 128-query half of the unit against a pair of 128-entry tiles, written by ONE N = 256
    // MMA per K step instead of two N = 128 MMAs (one per query half).  Issuer i takes query
    // half i of every tile pair; TMEM use, the epilogue's loads per warp and the code words are
    // unchanged.  Measured at c2: 13.10 -> 12.6 ms, the MMA issue sitting on the hand-off chain.
    constexpr bool PAIR = ONEPASS && !F8 && C::kTPS >= 2;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sB = smem;
    uint8_t *sA = smem + C::kStages * C::kStageBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + C::kBarOff);
    uint64_t *b_full = bars, *b_empty = bars + C::kStages;
    uint64_t *a_full = bars + 2 * C::kStages, *a_empty = a_full + 2;
    uint64_t *acc_full = a_empty + 2, *acc_empty = acc_full + 2, *drain = acc_empty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + kIssuers);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::kStages; ++i) {
            mbar_init(smem_u32(&b_full[i]), 1);
            // one arrival per tile of the stage (FP8: per tile and epilogue warp reading it; the
            // one-pass form's epilogue gives each tile to half the epilogue warps)
            mbar_init(smem_u32(&b_empty[i]), F8 ? C::kTPS * (ONEPASS ? kEpiWarps / 2 : kEpiWarps) : C::kTPS);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&a_full[i]), 1);
            mbar_init(smem_u32(&a_empty[i]), kIssuers);  // every issuer commits at the end of a unit
            mbar_init(smem_u32(&acc_full[i]), 1);
            // one elected arrive per epilogue warp reading the buffer (one-pass form: half of them)
            mbar_init(smem_u32(&acc_empty[i]), ONEPASS ? kEpiWarps / 2 : kEpiWarps);
        }
        for (int i = 0; i < kIssuers; ++i) mbar_init(smem_u32(&drain[i]), 1);
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

    if (REG) {
        // every thread of each warpgroup: warps 0-3 give registers back, warps 4-19 take them
        if (warp < kEpiWarp0) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegLow));
        else asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegHigh));
    }
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t stage = 0, sphase = 0, abuf = 0, aphase = 0;
            int64_t b_issued = 0, a_issued = 0;  // copies issued into the B ring / A buffers
            bool ok = true;
            for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
                const DenseGroup &gr = MULTI ? group_of(p, u) : p.g;
                const int64_t qt = (u - gr.unit0) % gr.n_qt, ch = (u - gr.unit0) / gr.n_qt;
                const int64_t t0 = ch * gr.tiles_per_chunk, t1 = min64(gr.n_tiles, t0 + gr.tiles_per_chunk);
                if (!(ok = mbar_wait(smem_u32(&a_empty[abuf]), aphase ^ 1, abort_flag, p.wait_ns))) break;
                mbar_arrive_expect_tx(smem_u32(&a_full[abuf]), C::kA);
                bulk_g2s(smem_u32(sA + abuf * C::kA), static_cast<const char *>(gr.qpre) + qt * C::kA, C::kA,
                         smem_u32(&a_full[abuf]));
                ++a_issued;
                if (++abuf == 2) { abuf = 0; aphase ^= 1; }
                for (int64_t tt = t0; tt < t1; tt += C::kTPS) {
                    const uint32_t bytes = (uint32_t)min64(C::kTPS, t1 - tt) * C::kB;
                    if (!(ok = mbar_wait(smem_u32(&b_empty[stage]), sphase ^ 1, abort_flag, p.wait_ns))) break;
                    mbar_arrive_expect_tx(smem_u32(&b_full[stage]), bytes);
                    bulk_g2s(smem_u32(sB + stage * C::kStageBytes), static_cast<const char *>(gr.pre) + tt * C::kB,
                             bytes, smem_u32(&b_full[stage]));
                    ++b_issued;
                    if (++stage == C::kStages) { stage = 0; sphase ^= 1; }
                }
                // failure-path test: the next unit's query copy never comes, so the MMA
                // warps' wait for it runs out and the CTA takes the abort path
                if (p.stall) break;
            }
            // copies still in flight must land before this CTA's shared memory goes away:
            // slot s last received copy number c = s + kStages * lap, lap = (issued - 1 - s) / kStages,
            // which completes phase `lap` of its barrier (parity lap & 1)
            for (int s = 0; s < C::kStages; ++s)
                if (b_issued > s)
                    mbar_drain(smem_u32(&b_full[s]), (uint32_t)(((b_issued - 1 - s) / C::kStages) & 1), kWaitLimitNs);
            for (int s = 0; s < 2; ++s)
                if (a_issued > s) mbar_drain(smem_u32(&a_full[s]), (uint32_t)(((a_issued - 1 - s) / 2) & 1), kWaitLimitNs);
        }
    } else if (warp <= kIssuers) {
        // ------------------------------------------------------------ MMA issuers
        // Issuer i handles the tiles with (tile counter % 2) == i, always into
        // accumulator buffer i (256 columns: A tile `sub` in columns 128*sub ..).
        if (lane == 0) {
            const uint32_t me = (uint32_t)(warp - 1);
            // BF16 operands (FP8: e4m3 operands), FP32 accumulator
            constexpr uint32_t idesc = F8 ? idesc_e4m3_f32(kTileQ, kDE) : idesc_bf16_f32(kTileQ, kDE);
            uint32_t stage = 0, sphase = 0, abuf = 0, aphase = 0, uses = 0;
            uint64_t g = 0;  // tile counter of this CTA
            bool ok = true;
            for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
                const DenseGroup &gr = MULTI ? group_of(p, u) : p.g;
                const int64_t ch = (u - gr.unit0) / gr.n_qt;
                const int64_t t0 = ch * gr.tiles_per_chunk, t1 = min64(gr.n_tiles, t0 + gr.tiles_per_chunk);
                if (!(ok = mbar_wait(smem_u32(&a_full[abuf]), aphase, abort_flag, p.wait_ns))) break;
                tc_fence_after();
                const uint32_t a_addr = smem_u32(sA + abuf * C::kA);
                for (int64_t tt = t0; ok && tt < t1; tt += C::kTPS) {
                    const int nt = (int)min64(C::kTPS, t1 - tt);
                    // wait for every fill of the ring, even one holding none of this issuer's
                    // tiles, so that the parity of the next wait on the slot cannot alias
                    if (!(ok = mbar_wait(smem_u32(&b_full[stage]), sphase, abort_flag, p.wait_ns))) break;
                    if (PAIR) {
                        constexpr uint32_t idesc2 = idesc_bf16_f32(kTileQ, 2 * kDE);
                        for (int j = 0; j < nt; j += 2) {
                            if (!(ok = mbar_wait(smem_u32(&acc_empty[me]), (uses & 1) ^ 1, abort_flag, p.wait_ns))) break;
                            tc_fence_after();
                            const uint32_t b_addr = smem_u32(sB + stage * C::kStageBytes + j * C::kB);
#pragma unroll
                            for (int kk = 0; kk < KP / 16; ++kk) {
                                const uint64_t ad = smem_desc(a_addr + me * kTileQ * KP * 2 + kk * 256, 128, KP * 16);
                                const uint64_t bd = smem_desc(b_addr + kk * 256, 128, KP * 16);
                                umma_bf16(tmem + me * 256, ad, bd, idesc2, kk > 0 ? 1u : 0u);
                            }
                            umma_commit(smem_u32(&acc_full[me]));
                            ++uses;
                        }
                        g += nt;
                    } else {
                        for (int j = 0; j < nt; ++j, ++g) {
                            if ((uint32_t)(g & 1) != me) continue;
                            if (!(ok = mbar_wait(smem_u32(&acc_empty[me]), (uses & 1) ^ 1, abort_flag, p.wait_ns))) break;
                            tc_fence_after();
                            const uint32_t b_addr = smem_u32(sB + stage * C::kStageBytes + j * C::kB);
#pragma unroll
                            for (int sub = 0; sub < kDQ / kTileQ; ++sub) {
#pragma unroll
                                for (int kk = 0; kk < KP / 16; ++kk) {
                                    // A: two core matrices along K, 128 B apart (BF16: 16 columns; FP8: the hi
                                    // and lo bytes of 16 columns); 8-row groups KP*16 B apart; A tile `sub` =
                                    // query rows 128*sub .. 128*sub+127
                                    const uint64_t ad = smem_desc(a_addr + sub * kTileQ * KP * 2 + kk * 256, 128, KP * 16);
                                    if (F8) {
                                        // entry side: the core matrix of columns 16kk.. read twice (K stride 0)
                                        const uint64_t bd = smem_desc(b_addr + kk * 128, 0, KP * 8);
                                        umma_f8(tmem + me * 256 + sub * kDE, ad, bd, idesc, kk > 0 ? 1u : 0u);
                                    } else {
                                        const uint64_t bd = smem_desc(b_addr + kk * 256, 128, KP * 16);
                                        umma_bf16(tmem + me * 256 + sub * kDE, ad, bd, idesc, kk > 0 ? 1u : 0u);
                                    }
                                }
                            }
                            umma_commit(smem_u32(&acc_full[me]));
                            ++uses;
                        }
                    }
                    if (++stage == C::kStages) { stage = 0; sphase ^= 1; }
                }
                if (!ok) break;
                umma_commit(smem_u32(&a_empty[abuf]));
                if (++abuf == 2) { abuf = 0; aphase ^= 1; }
            }
            // every MMA issued so far must finish before TMEM is released
            umma_commit(smem_u32(&drain[me]));
            mbar_drain(smem_u32(&drain[me]), 0, kWaitLimitNs);
        }
    } else if (warp < kEpiWarp0) {
        // idle: completes the first warpgroup
    } else if (ONEPASS) {
        // ------------------------------------------------------------ epilogue, one-pass form
        // Two warp groups, one per accumulator buffer: while one group reduces its tile, the
        // other loads the next, so the TMEM loads and the max trees of an SM sub-partition
        // overlap instead of running in lockstep.  Every work unit holds an even number of
        // entry tiles (the host makes tiles_per_chunk even; n_tiles is even), so every unit
        // starts on buffer 0 and group `grp` takes tiles j = grp, grp + 2, ... of each unit,
        // always in buffer grp.  Warp (group, A tile, TMEM lane quarter) reads all 128 entry
        // columns of its 32 query rows (two 64-column loads), so it forms the four group
        // codes of the tile -- one word per (query, tile) -- and the best group it has seen
        // in the chunk (candidate slot 2 chunk + group).
        // FP8: the group's largest raw accumulator A bounds its scores u_i = RN(acc_i s_i/256
        // + b_i) from above by max(RU(A smax + bmax), RU(A smin + bmax)) with the group's scale
        // range and largest error term (k_f8_group_bounds).
        const int ew = warp - kEpiWarp0;
        const int quarter = warp & 3;             // TMEM lanes this warp may read: 32*quarter ..
        const int grp = ew >> 3;                  // accumulator buffer this warp serves
        const int sub = (ew >> 2) & 1;
        // PAIR: buffer grp = query half grp, columns 128*sub .. = tile 2p + sub of the pair;
        // otherwise buffer grp = tile parity grp, columns 128*sub .. = query half sub
        const int qh = PAIR ? grp : sub;          // query half of this warp's rows
        const int tp = PAIR ? sub : grp;          // tile parity this warp reads
        const int row = qh * kTileQ + quarter * 32 + lane;
        const bool releaser = (ew & 7) == 0 && lane == 0;  // hands this group's B stages back
        const uint32_t taddr = tmem + grp * 256 + sub * kDE + ((uint32_t)(quarter * 32) << 16);
        const uint32_t full_bar = smem_u32(&acc_full[grp]), empty_bar = smem_u32(&acc_empty[grp]);
        uint32_t uses = 0;  // tiles this group has taken: use number of its buffer
        int unit_stage = 0; // ring stage of the current unit's first tile
        bool ok = true;
        for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
            const DenseGroup &gr = MULTI ? group_of(p, u) : p.g;
            const int64_t qt = (u - gr.unit0) % gr.n_qt, ch = (u - gr.unit0) / gr.n_qt;
            const int32_t t0 = (int32_t)(ch * gr.tiles_per_chunk);
            const int32_t nt_u = (int32_t)min64(gr.n_tiles - t0, gr.tiles_per_chunk);  // even
            const int64_t q = qt * kDQ + row;
            const bool qvalid = q < gr.nq;
            const int64_t wstride = gr.n_qt * kDQ;  // words between consecutive tiles of a query
            float best = -INFINITY;
            int32_t bgid = -1;  // the 32-entry group of `best`
            uint32_t *gb = gr.gbits + ch * gr.words * wstride + q + tp * wstride;
            const int32_t n32 = (int32_t)gr.n;
            const float inv = gr.code_inv, base = p.code_base;
            // tile j sits in slot j % kTPS of stage unit_stage + j / kTPS (mod kStages)
            int slot = tp % C::kTPS;
            int stage = unit_stage + tp / C::kTPS;
            if (stage >= C::kStages) stage -= C::kStages;
            for (int32_t j = tp; j < nt_u; j += 2, gb += 2 * wstride) {
                // the warp leaves together: its TMEM loads and hand-offs below are warp-wide
                ok = __all_sync(0xffffffffu, mbar_wait(full_bar, uses & 1u, abort_flag, p.wait_ns));
                if (!ok) break;
                ++uses;
                tc_fence_after();
                // this tile's MMAs are done with the stage; the unit's last tile also arrives
                // for the slots its (short) stage did not fill
                // PAIR: each query half's releaser (tile parity 0) arrives once per pair, and at
                // the unit's last pair also for the pairs its (short) stage did not hold
                const uint32_t rel = PAIR ? (j + 2 >= nt_u ? (uint32_t)(1 + (C::kTPS - slot - 2) / 2) : 1u)
                                          : (j == nt_u - 1 ? (uint32_t)(C::kTPS - slot) : 1u);
                if (!F8 && releaser) mbar_arrive_cnt(smem_u32(&b_empty[stage]), rel);
                // group maxima straight from the loads (the values themselves are not needed).
                // One load per iteration of a loop that is not unrolled: the scratch registers
                // of a load are then free again before the next load is issued.
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                if (REG) {
                    // two loads in flight (64 scratch registers) per iteration
#pragma unroll 1
                    for (int i = 0; i < 2; ++i) {
                        float m0, m1;
                        tmem_ldmax2x32(taddr + 64 * i, m0, m1);
                        s0 = s2;
                        s1 = s3;
                        s2 = m0;
                        s3 = m1;
                    }
                } else {
#pragma unroll 1
                    for (int i = 0; i < 4; ++i) {
                        const float mi = tmem_ldmax32(taddr + 32 * i);
                        s0 = s1;
                        s1 = s2;
                        s2 = s3;
                        s3 = mi;
                    }
                }
                // the maxima are in registers: hand the accumulator back to the MMA warp now
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(empty_bar);
                if (F8) {
                    const float4 *gbd = reinterpret_cast<const float4 *>(smem + stage * C::kStageBytes +
                                                                         slot * C::kB + f8_group_off(KP));
                    const float4 b0 = gbd[0], b1 = gbd[1], b2 = gbd[2], b3 = gbd[3];
                    __syncwarp();
                    if (lane == 0) mbar_arrive_cnt(smem_u32(&b_empty[stage]), rel);
                    s0 = fmaxf(__fmaf_ru(s0, b0.x, b0.z), __fmaf_ru(s0, b0.y, b0.z));
                    s1 = fmaxf(__fmaf_ru(s1, b1.x, b1.z), __fmaf_ru(s1, b1.y, b1.z));
                    s2 = fmaxf(__fmaf_ru(s2, b2.x, b2.z), __fmaf_ru(s2, b2.y, b2.z));
                    s3 = fmaxf(__fmaf_ru(s3, b3.x, b3.z), __fmaf_ru(s3, b3.y, b3.z));
                }
                // threshold candidate: the best group (lowest on ties) holding a real entry;
                // after the first tiles of a chunk the test rarely passes
                const float m = fmax3(s0, s1, fmaxf(s2, s3));
                if (m > best) {
                    const int32_t gid = (t0 + j) * 4 + (s0 == m ? 0 : s1 == m ? 1 : s2 == m ? 2 : 3);
                    if (gid * 32 < n32) {
                        best = m;
                        bgid = gid;
                    }
                }
                // the tile's word: codes of groups 0-3 (byte i = group i), taken from the low
                // byte of each 2^23 + code float by byte permutes.  The upper clamp only acts
                // when the tile's largest code would pass 255 (never for scores within the norm
                // bound); a streaming store, so that the map does not evict the prefix from L2
                if (CODES) {
                    uint32_t c0 = code_bits_unclamped(s0, inv, base), c1 = code_bits_unclamped(s1, inv, base);
                    uint32_t c2 = code_bits_unclamped(s2, inv, base), c3 = code_bits_unclamped(s3, inv, base);
                    if (code_bits_unclamped(m, inv, base) > kCodeBits0 + 255u) {
                        c0 = min(c0, kCodeBits0 + 255u);
                        c1 = min(c1, kCodeBits0 + 255u);
                        c2 = min(c2, kCodeBits0 + 255u);
                        c3 = min(c3, kCodeBits0 + 255u);
                    }
                    __stcs(gb, __byte_perm(__byte_perm(c0, c1, 0x0040), __byte_perm(c2, c3, 0x0040), 0x5410));
                }
                slot += 2;
                while (slot >= C::kTPS) {
                    slot -= C::kTPS;
                    if (++stage == C::kStages) stage = 0;
                }
            }
            if (!ok) break;
            unit_stage = (int)((unit_stage + (nt_u + C::kTPS - 1) / C::kTPS) % C::kStages);
            // one writer per (query, chunk, group): every slot written
            if (qvalid) gr.cand[q * (2 * gr.chunks) + 2 * ch + tp] = bgid >= 0 ? pack_best(best, (uint32_t)bgid) : 0ull;
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - kEpiWarp0;         // 0 .. kEpiWarps-1
        const int quarter = warp & 3;            // TMEM lanes this warp may read: 32*quarter ..
        const int seg = ew >> 2;                 // accumulator columns 64*seg .. 64*seg + 63
        const int sub = seg >> 1;                // query A tile of those columns
        const int half = seg & 1;                // entry half of the B tile: entries 64*half ..
        const int row = sub * kTileQ + quarter * 32 + lane;
        const bool releaser = ew == 0 && lane == 0;  // hands B stages back to the producer
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        uint32_t stage = 0, sphase = 0;
        uint32_t g = 0;  // tile counter of this CTA: buffer g & 1, its use number g >> 1
        bool ok = true;
        for (int64_t u = blockIdx.x; ok && u < p.n_units; u += G) {
            const DenseGroup &gr = MULTI ? group_of(p, u) : p.g;
            const int64_t qt = (u - gr.unit0) % gr.n_qt, ch = (u - gr.unit0) / gr.n_qt;
            // tile and entry numbers fit in 32 bits (n < 2^31 - 256 is enforced by hn_index_build)
            const int32_t t0 = (int32_t)(ch * gr.tiles_per_chunk);
            const int32_t t1 = (int32_t)min64(gr.n_tiles, (int64_t)t0 + gr.tiles_per_chunk);
            const int64_t q = qt * kDQ + row;
            const bool qvalid = q < gr.nq;
            const float thr = (PHASE == 2 && qvalid) ? gr.tau[q] : INFINITY;

            uint32_t gword = 0;  // PHASE 2: passing-group bits of the current 16 tiles
            uint32_t *gb = PHASE == 2 ? gr.gbits + (ch * 2 + half) * gr.words * (gr.n_qt * kDQ) + q
                                                      : nullptr;
            const int32_t n32 = (int32_t)gr.n;
            int32_t e0 = t0 * kDE + half * 64;    // first entry of this warp's 64 columns
            for (int32_t tt = t0; ok && tt < t1; tt += C::kTPS) {
                const int nt = t1 - tt < C::kTPS ? t1 - tt : C::kTPS;
                for (int j = 0; j < nt; ++j, ++g, e0 += kDE) {
                    const uint32_t buf = g & 1u;
                    // the warp leaves together: its TMEM loads and hand-offs below are warp-wide
                    ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_full[buf]), (g >> 1) & 1u, abort_flag,
                                                           p.wait_ns));
                    if (!ok) break;
                    tc_fence_after();
                    // this tile's MMAs are done with the stage; the last tile of a short stage
                    // also arrives for the tiles the stage did not hold
                    const uint32_t rel = j == nt - 1 ? 1 + C::kTPS - nt : 1;
                    if (!F8 && releaser) mbar_arrive_cnt(smem_u32(&b_empty[stage]), rel);
                    const int32_t t = tt + j;
                    // FP8: this warp's 64 per-entry scales / error terms in the stage
                    const uint8_t *esc = smem + stage * C::kStageBytes + j * C::kB + (F8 ? f8_scale_off(KP) : 0);
                    if (PHASE == 2 && !F8) {
                        // BF16 Phase 2 compares raw group maxima with tau_q: the reducing loads
                        // return the two 32-entry maxima of this warp's 64 columns directly
                        float g0, g1;
                        tmem_ldmax2x32(tmem + buf * 256 + seg * 64 + lane_addr, g0, g1);
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
                        const int32_t ti = t - t0;
                        gword |= ((g0 >= thr ? 1u : 0u) | (g1 >= thr ? 2u : 0u)) << (2 * (ti & 15));
                        if ((ti & 15) == 15 || t == t1 - 1) {
                            gb[(int64_t)(ti >> 4) * (gr.n_qt * kDQ)] = gword;
                            gword = 0;
                        }
                    } else {
                        float v[64];
                        tmem_ld64(tmem + buf * 256 + seg * 64 + lane_addr, v);
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(&acc_empty[buf]));
                        if (F8) {
                            // u = fma(acc, s_i / 256, b_i): one rounding, packed pairs
                            const float4 *s4 = reinterpret_cast<const float4 *>(esc) + half * 16;
                            const float4 *b4 = reinterpret_cast<const float4 *>(esc + kF8Tile * 4) + half * 16;
#pragma unroll
                            for (int i = 0; i < 16; ++i) {
                                const float4 sv = s4[i], bv = b4[i];
                                const float2 lo = __ffma2_rn(make_float2(v[4 * i], v[4 * i + 1]), make_float2(sv.x, sv.y),
                                                             make_float2(bv.x, bv.y));
                                const float2 hi = __ffma2_rn(make_float2(v[4 * i + 2], v[4 * i + 3]),
                                                             make_float2(sv.z, sv.w), make_float2(bv.z, bv.w));
                                v[4 * i] = lo.x;
                                v[4 * i + 1] = lo.y;
                                v[4 * i + 2] = hi.x;
                                v[4 * i + 3] = hi.y;
                            }
                            __syncwarp();
                            if (lane == 0) mbar_arrive_cnt(smem_u32(&b_empty[stage]), rel);
                        }
                        if (PHASE == 3) {
                            // verification: every score of the Phase-2 arithmetic to memory
                            if (qvalid) {
                                float *d = p.dump + q * gr.n;
                                for (int i = 0; i < 64; ++i)
                                    if (e0 + i < n32) d[e0 + i] = v[i];
                            }
                            continue;
                        }
                        // bit 2 (tile mod 16) + k: the maximum of the 32 scores 32k .. 32k + 31 reaches
                        // tau_q.  The bits go out as one coalesced word per 16 tiles; k_dense_extract
                        // finds the survivors of those groups.  Nothing here waits on memory: the
                        // accumulator hand-off has no slack for a rare, slow path in any warp.
                        const int32_t ti = t - t0;
                        const float g0 = fmaxf(max16(v), max16(v + 16)), g1 = fmaxf(max16(v + 32), max16(v + 48));
                        gword |= ((g0 >= thr ? 1u : 0u) | (g1 >= thr ? 2u : 0u)) << (2 * (ti & 15));
                        if ((ti & 15) == 15 || t == t1 - 1) {
                            gb[(int64_t)(ti >> 4) * (gr.n_qt * kDQ)] = gword;
                            gword = 0;
                        }
                    }
                }
                if (++stage == C::kStages) { stage = 0; sphase ^= 1; }
            }
            if (!ok) break;
        }
    }

    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status + ST_TIMEOUT, 1);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------ Phase-2 survivors
// Second step of the dense Phase 2.  Every 32-entry group whose maximum reached tau_q in
// the tensor-core scan (one bit of gbits) is scored again on the CUDA cores with the
// stream scan's arithmetic: an FP32 FMA chain over the stored prefix in column order
// (BF16 index: the BF16 values against the BF16-rounded query; FP8 index: s_i x^ against
// the exact query, then + b_i).  The query slack E_q bounds that arithmetic as well as
// the tensor cores', so keeping the entries with score >= tau_q keeps every possible
// answer.  A block takes 256 queries and one entry chunk (many warps in flight hide the
// gathers); a warp scores one group at a time, one entry a lane, and takes the group's
// survivor slots with one atomicAdd on the query's count.
struct ExtractParams {
    const void *pre;          // BF16 prefix (UMMA order) or FP8 tiles
    const float *qpre32;      // [nq][kp] query prefix in the scan precision
    const uint32_t *gbits;    // as written by k_dense_scan
    int64_t n, n_tiles, nq, q_pad, tiles_per_chunk, chunks, words;
    const float *tau;
    int32_t *bucket, *count;  // count: slots already used (soft mode: the kept best); may pass cap
    int32_t cap;
    float code_inv, code_base;  // one-pass form: the group code of k_dense_scan<., 4, .>
    long long *counters;        // device counters (CT_GROUPS: groups scored)
};

// One entry of a flagged group: its stored prefix (and FP8 scale and error term), and the
// CUDA-core score the extraction kernels and the verification kernel compute from it.
template <int KP, bool F8>
struct GroupEntry {
    static constexpr int kV = F8 ? KP / 16 : KP / 8;  // 16-byte pieces of the stored prefix
    uint4 v[kV];
    float esc, b;                                      // FP8: s_i (exact) and b_i

    __device__ __forceinline__ void load(const ExtractParams &x, int64_t e) {
        if (F8) {
            const uint8_t *tile8 = static_cast<const uint8_t *>(x.pre) + (e >> 7) * kF8TileBytes(KP);
            const float *sc2 = reinterpret_cast<const float *>(tile8 + f8_scale_off(KP));
#pragma unroll
            for (int i = 0; i < kV; ++i) v[i] = *reinterpret_cast<const uint4 *>(tile8 + umma8_offset(e & 127, 16 * i, KP));
            esc = sc2[e & 127] * kF8QScale;
            b = sc2[kF8Tile + (e & 127)];
        } else {
#pragma unroll
            for (int i = 0; i < kV; ++i)
                v[i] = *reinterpret_cast<const uint4 *>(static_cast<const char *>(x.pre) + pre16_offset(e, 8 * i, KP));
        }
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < kV; ++i) v[i] = make_uint4(0u, 0u, 0u, 0u);
        esc = 0.f;
        b = 0.f;
    }
    // FP32 FMA chain over the prefix columns in order (BF16: the stored values against the
    // BF16-rounded query; FP8: s_i x^ against the exact query, then + b_i)
    __device__ __forceinline__ float score(const float *qp) const {
        float s = 0.f;
        if (F8) {
#pragma unroll
            for (int i = 0; i < kV; ++i) {
                const __nv_fp8x2_storage_t *h = reinterpret_cast<const __nv_fp8x2_storage_t *>(&v[i]);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(h[u], __NV_E4M3)));
                    s = fmaf(qp[16 * i + 2 * u], f.x * esc, s);
                    s = fmaf(qp[16 * i + 2 * u + 1], f.y * esc, s);
                }
            }
            s += b;
        } else {
#pragma unroll
            for (int i = 0; i < kV; ++i) {
                const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v[i]);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float2 f = __bfloat1622float2(h[u]);
                    s = fmaf(qp[8 * i + 2 * u], f.x, s);
                    s = fmaf(qp[8 * i + 2 * u + 1], f.y, s);
                }
            }
        }
        return s;
    }
};

template <int KP, bool F8>
__device__ __forceinline__ float group_entry_score(const ExtractParams &x, int64_t e, const float *qp) {
    GroupEntry<KP, F8> g;
    g.load(x, e);
    return g.score(qp);
}

template <int KP, bool F8>
__global__ void __launch_bounds__(256) k_dense_extract(const ExtractParams x) {
    const int lane = threadIdx.x & 31;
    uint32_t scored = 0;  // groups this warp scored (warp-uniform)
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // this thread's query
    const bool qv = q < x.nq;
    const float tau = qv ? x.tau[q] : INFINITY;
    {
        const int64_t c = blockIdx.y;  // this block's entry chunk
        const int64_t t0 = c * x.tiles_per_chunk;
        const int64_t nt = min64(x.n_tiles - t0, x.tiles_per_chunk);
        const int64_t nw = (nt + 15) / 16;
        for (int h = 0; h < 2; ++h) {
            const uint32_t *gw = x.gbits + (c * 2 + h) * x.words * x.q_pad;
            for (int64_t w0 = 0; w0 < nw; w0 += 8) {
                // 8 independent coalesced loads in flight; most words are zero
                uint32_t wv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) wv[i] = (qv && w0 + i < nw) ? gw[(w0 + i) * x.q_pad + q] : 0u;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                const uint32_t word = wv[i];
                const int64_t w = w0 + i;
                unsigned pend = __ballot_sync(0xffffffffu, word != 0u);
                while (pend) {
                    const int o = __ffs(pend) - 1;
                    pend &= pend - 1;
                    uint32_t wo = __shfl_sync(0xffffffffu, word, o);
                    const float to = __shfl_sync(0xffffffffu, tau, o);
                    const int64_t qo = q - lane + o;
                    const float *qp = x.qpre32 + qo * KP;
                    while (wo) {
                        const int b = __ffs(wo) - 1;
                        wo &= wo - 1;
                        ++scored;
                        const int64_t e = (t0 + w * 16 + (b >> 1)) * kDE + h * 64 + (b & 1) * 32 + lane;
                        const bool hit = e < x.n && group_entry_score<KP, F8>(x, e, qp) >= to;
                        const unsigned hb = __ballot_sync(0xffffffffu, hit);
                        if (hb) {
                            int base = 0;
                            if (lane == o) base = atomicAdd(x.count + qo, __popc(hb));
                            base = __shfl_sync(0xffffffffu, base, o);
                            if (hit) {
                                const int slot = base + __popc(hb & ((1u << lane) - 1u));
                                if (slot < x.cap) x.bucket[qo * x.cap + slot] = (int32_t)e;
                            }
                        }
                    }
                }
                }
            }
        }
    }
    if (lane == 0 && scored) atomicAdd(reinterpret_cast<unsigned long long *>(x.counters + CT_GROUPS), scored);
}

// The same step for the one-pass form: the map holds one word per (query, tile) with
// the 8-bit codes of the tile's four 32-entry groups' largest scores, and a group is
// scored when its code reaches code(tau_q) (a non-decreasing code, so every group whose
// largest score reaches tau_q is among them); __vcmpgeu4 tests the four codes of a word
// at once.  The words are read with the streaming hint, so that the map (read once)
// leaves the prefix, which the visited groups gather, in L2.
// Six blocks (48 warps) per SM: more gathers in flight than the register-limited five
// (measured at c2, BF16: 8.41 -> 7.93 ms; eight blocks spill and take 8.23 ms)
template <int KP, bool F8>
__global__ void __launch_bounds__(256, 6) k_dense_extract_codes(const ExtractParams x) {
    const int lane = threadIdx.x & 31;
    uint32_t scored = 0;  // groups this warp scored (warp-uniform)
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // this thread's query
    const bool qv = q < x.nq;
    const float tau = qv ? x.tau[q] : INFINITY;
    const uint32_t ct4 = code_threshold(tau, x.code_inv, x.code_base) * 0x01010101u;
    const int64_t c = blockIdx.y;  // this block's entry chunk
    const int64_t t0 = c * x.tiles_per_chunk;
    const int64_t nt = min64(x.n_tiles - t0, x.tiles_per_chunk);
    const uint32_t *gw = x.gbits + c * x.words * x.q_pad;
    for (int64_t w0 = 0; w0 < nt; w0 += 8) {
        // 8 independent coalesced loads in flight; most codes fail
        uint32_t wv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) wv[i] = (qv && w0 + i < nt) ? __ldcs(gw + (w0 + i) * x.q_pad + q) : 0u;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t w = w0 + i;  // the tile t0 + w
            // the top bit of every passing code's byte; absent words pass nothing
            const uint32_t word = (qv && w < nt) ? (__vcmpgeu4(wv[i], ct4) & 0x80808080u) : 0u;
            unsigned pend = __ballot_sync(0xffffffffu, word != 0u);
            while (pend) {
                const int o = __ffs(pend) - 1;
                pend &= pend - 1;
                uint32_t wo = __shfl_sync(0xffffffffu, word, o);
                const float to = __shfl_sync(0xffffffffu, tau, o);
                const int64_t qo = q - lane + o;
                const float *qp = x.qpre32 + qo * KP;
                while (wo) {
                    const int b = (__ffs(wo) - 1) >> 3;  // code byte = group of the tile
                    wo &= wo - 1;
                    ++scored;
                    const int64_t e = (t0 + w) * kDE + b * 32 + lane;
                    const bool hit = e < x.n && group_entry_score<KP, F8>(x, e, qp) >= to;
                    const unsigned hb = __ballot_sync(0xffffffffu, hit);
                    if (hb) {
                        int base = 0;
                        if (lane == o) base = atomicAdd(x.count + qo, __popc(hb));
                        base = __shfl_sync(0xffffffffu, base, o);
                        if (hit) {
                            const int slot = base + __popc(hb & ((1u << lane) - 1u));
                            if (slot < x.cap) x.bucket[qo * x.cap + slot] = (int32_t)e;
                        }
                    }
                }
            }
        }
    }
    if (lane == 0 && scored) atomicAdd(reinterpret_cast<unsigned long long *>(x.counters + CT_GROUPS), scored);
}

// Verification: the CUDA-core score of every (query, entry) pair, computed by
// group_entry_score -- the arithmetic of k_dense_extract and of the stream scan's
// FMA chain over the same stored prefix.  One thread per pair.
template <int KP, bool F8>
__global__ void __launch_bounds__(256) k_fma_scores(const ExtractParams x, float *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= x.nq * x.n) return;
    const int64_t q = i / x.n, e = i % x.n;
    out[i] = group_entry_score<KP, F8>(x, e, x.qpre32 + q * KP);
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

// About `upc` work units per CTA (autotuned, 32 by default), numbered chunk-major
// so that the running CTAs share entry tiles in L2.
static void dense_chunking(int64_t n_tiles, int64_t n_qt, int G, int upc, int64_t *tiles_per_chunk, int64_t *chunks) {
    int64_t c = ((int64_t)upc * G + n_qt - 1) / n_qt;
    c = max64(1, min64(c, n_tiles));
    const int64_t tpc = (n_tiles + c - 1) / c;
    *tiles_per_chunk = tpc;
    *chunks = (n_tiles + tpc - 1) / tpc;
}

int64_t dense_cand_slots(const Index &ix, int64_t nq) {
    int64_t tpc = 0, chunks = 0;
    dense_chunking(ix.n_tiles * (kTileE / kDE), (nq + kDQ - 1) / kDQ, num_sms(), ix.units_per_cta, &tpc, &chunks);
    return 2 * chunks;
}

bool dense_scan_supported(const Index &ix) {
    return (ix.prefix == HN_PREFIX_BF16 || ix.prefix == HN_PREFIX_FP8_E4M3) &&
           (ix.k_pad16 == 16 || ix.k_pad16 == 32 || ix.k_pad16 == 64);
}

template <int KP, int PHASE, bool F8>
static int dense_smem() {
    using C = DenseCfg<KP, PHASE, F8>;
    return (int)C::kSmem < kMinDenseSmem ? kMinDenseSmem : (int)C::kSmem;
}

template <int KP, int PHASE, bool F8>
static cudaError_t set_attr1() {
    return cudaFuncSetAttribute(k_dense_scan<KP, PHASE, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                dense_smem<KP, PHASE, F8>());
}

template <int KP, bool F8>
static cudaError_t set_attr2() {
    cudaError_t e = set_attr1<KP, 2, F8>();
    if (e == cudaSuccess) e = set_attr1<KP, 3, F8>();
    if (e == cudaSuccess) e = set_attr1<KP, 4, F8>();
    if (e == cudaSuccess) e = set_attr1<KP, 1, F8>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dense_scan<KP, 1, F8, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dense_smem<KP, 1, F8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dense_scan<KP, 4, F8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dense_smem<KP, 4, F8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dense_scan<KP, 4, F8, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dense_smem<KP, 4, F8>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_dense_scan<KP, 4, F8, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dense_smem<KP, 4, F8>());
    return e;
}

// The register-split one-pass epilogue (PHASE 4, or PHASE 1 without codes) is launched only
// if its threads are launched with exactly kRegLaunch registers: the split's increases draw
// on that launch budget.
template <int KP, int PHASE, bool F8, bool MULTI>
static bool reg_split_ok() {
    static int ok = -1;
    if (ok < 0) {
        cudaFuncAttributes a{};
        ok = cudaFuncGetAttributes(&a, k_dense_scan<KP, PHASE, F8, MULTI, true>) == cudaSuccess &&
             a.numRegs == kRegLaunch && a.maxThreadsPerBlock >= kDenseThreads;
    }
    return ok == 1;
}

template <int KP, int PHASE, bool F8>
static void launch_onepass_kernel(const DenseParams &p, int grid, cudaStream_t st) {
    if (!p.plain && reg_split_ok<KP, PHASE, F8, false>())
        k_dense_scan<KP, PHASE, F8, false, true><<<grid, kDenseThreads, dense_smem<KP, PHASE, F8>(), st>>>(p);
    else
        k_dense_scan<KP, PHASE, F8><<<grid, kDenseThreads, dense_smem<KP, PHASE, F8>(), st>>>(p);
}

// Kernel attributes for every instantiation; called once before the first launch
// (and before any stream capture, where attribute changes do not belong).
cudaError_t dense_init() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady) {
        cudaError_t e = set_attr2<16, false>();
        if (e == cudaSuccess) e = set_attr2<32, false>();
        if (e == cudaSuccess) e = set_attr2<64, false>();
        if (e == cudaSuccess) e = set_attr2<16, true>();
        if (e == cudaSuccess) e = set_attr2<32, true>();
        if (e == cudaSuccess) e = set_attr2<64, true>();
        num_sms();
        done = e;
    }
    return done;
}

template <int KP, bool F8>
static cudaError_t launch_kp(const DenseParams &p, int phase, int grid, cudaStream_t st) {
    cudaError_t e = dense_init();
    if (e != cudaSuccess) return e;
    switch (phase) {
        case 1: launch_onepass_kernel<KP, 1, F8>(p, grid, st); break;
        case 2: k_dense_scan<KP, 2, F8><<<grid, kDenseThreads, dense_smem<KP, 2, F8>(), st>>>(p); break;
        case 3: k_dense_scan<KP, 3, F8><<<grid, kDenseThreads, dense_smem<KP, 3, F8>(), st>>>(p); break;
        case 4: launch_onepass_kernel<KP, 4, F8>(p, grid, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KP>
static cudaError_t launch_kp_any(bool f8, const DenseParams &p, int phase, int grid, cudaStream_t st) {
    return f8 ? launch_kp<KP, true>(p, phase, grid, st) : launch_kp<KP, false>(p, phase, grid, st);
}

static cudaError_t launch_dense_kernel(int kp, bool f8, const DenseParams &p, int phase, int grid, cudaStream_t st) {
    switch (kp) {
        case 16: return launch_kp_any<16>(f8, p, phase, grid, st);
        case 32: return launch_kp_any<32>(f8, p, phase, grid, st);
        case 64: return launch_kp_any<64>(f8, p, phase, grid, st);
    }
    return cudaErrorNotSupported;
}

// Words of the group map the current search may use: what the workspace holds, or
// less when the search set a scratch limit (hn_search_opts.scratch_limit).
static int64_t map_cap(const Workspace &ws) {
    return ws.gbits_limit > 0 ? std::min(ws.gbits_limit, ws.gbits_cap) : ws.gbits_cap;
}

// Query tiles of the dense Phase-2 pass that starts at tile qt0: as many as fit the group
// bitmap's `cap` words (each pass is sized on its own: the chunking, and with it the word
// rounding, depends on the pass's tile count); 0 if even one tile does not fit.
static int64_t phase2_pass_tiles(int64_t n_tiles, int64_t n_qt, int64_t qt0, int G, int upc, int64_t cap);

// Words of the Phase-2 group bitmap for a pass over n_qt query tiles.
static int64_t gbits_words(int64_t n_tiles, int64_t n_qt, int G, int upc) {
    int64_t tpc = 0, chunks = 0;
    dense_chunking(n_tiles, n_qt, G, upc, &tpc, &chunks);
    return chunks * 2 * ((tpc + 15) / 16) * n_qt * kDQ;
}

// One-pass form: the chunking is that of the whole batch (so every pass writes the same
// candidate slots), and a query tile's codes take chunks * tpc * 256 words (a word per
// query and entry tile).  tpc is even, and so is n_tiles (rows are padded to 256), so
// every work unit holds an even number of tiles: the epilogue's two warp groups then
// take alternate tiles of every unit in a fixed order.
static int64_t onepass_tile_words(const Index &ix, int64_t n_qt_all, int64_t *tpc, int64_t *chunks) {
    const int64_t n_tiles = ix.n_tiles * (kTileE / kDE);
    dense_chunking(n_tiles, n_qt_all, num_sms(), ix.units_per_cta, tpc, chunks);
    *tpc = std::min(n_tiles, (*tpc + 1) & ~(int64_t)1);
    *chunks = (n_tiles + *tpc - 1) / *tpc;
    return *chunks * *tpc * kDQ;
}

// Candidate slots per query that the two-pass form's Phase 1 (the one-pass chunking) writes.
int64_t dense_phase1_slots(const Index &ix, int64_t nq) {
    int64_t tpc = 0, chunks = 0;
    onepass_tile_words(ix, (nq + kDQ - 1) / kDQ, &tpc, &chunks);
    return 2 * chunks;
}

// The one-pass epilogue's tile order needs even unit lengths.
static bool onepass_chunking_ok(const DenseGroup &g) {
    return g.n_tiles % 2 == 0 && g.tiles_per_chunk % 2 == 0 && g.tiles_per_chunk > 0;
}

// Chunking of a joined group: the group's own one-pass chunking, with at least
// kMultiMinTiles entry tiles a unit (many small groups share the SMs anyway).
constexpr int64_t kMultiMinTiles = 16;

static void multi_chunking(const Index &ix, int64_t nq, int64_t *tpc, int64_t *chunks) {
    const int64_t n_tiles = ix.n_tiles * (kTileE / kDE);
    onepass_tile_words(ix, (nq + kDQ - 1) / kDQ, tpc, chunks);
    *tpc = std::min(n_tiles, std::max(*tpc, kMultiMinTiles));
    *chunks = (n_tiles + *tpc - 1) / *tpc;
}

// Group-map words the workspace holds for nq queries: the whole batch up to 4 GiB (two-pass
// bits) or 16 GiB (one-pass codes), larger batches taking the scan in passes over query
// tiles; at most limit_bytes when that is > 0; always at least one query tile's.
int64_t dense_gbits_words(const Index &ix, int64_t nq, bool onepass, int64_t limit_bytes) {
    const int64_t n_tiles = ix.n_tiles * (kTileE / kDE);
    const int64_t n_qt = (nq + kDQ - 1) / kDQ;
    int64_t all, one, max_words;
    if (onepass) {
        int64_t tpc = 0, chunks = 0;
        one = onepass_tile_words(ix, n_qt, &tpc, &chunks);
        multi_chunking(ix, nq, &tpc, &chunks);  // a shared multi-index scan may chunk more coarsely
        one = std::max(one, chunks * tpc * kDQ);
        all = one * n_qt;
        max_words = (int64_t)1 << 32;
    } else {
        all = gbits_words(n_tiles, n_qt, num_sms(), ix.units_per_cta);
        one = gbits_words(n_tiles, 1, num_sms(), ix.units_per_cta);
        max_words = (int64_t)1 << 30;
    }
    int64_t w = std::min(all, max_words);
    if (limit_bytes > 0) w = std::min(w, limit_bytes / 4);
    return std::max(w, one);
}

static int64_t phase2_pass_tiles(int64_t n_tiles, int64_t n_qt, int64_t qt0, int G, int upc, int64_t cap) {
    int64_t nqt = n_qt - qt0;
    while (nqt > 1 && gbits_words(n_tiles, nqt, G, upc) > cap) nqt = (nqt + 1) / 2;
    return gbits_words(n_tiles, nqt, G, upc) > cap ? 0 : nqt;
}

// Kernel launches of the dense scan steps after query preparation: two-pass, one per
// Phase-1 scan plus a scan and an extraction per Phase-2 pass (the threshold kernel is
// counted by the caller); one-pass, a scan, a threshold and an extraction per pass.
int64_t dense_phase2_launches(const Index &ix, int64_t nq, bool onepass) {
    const int64_t n_qt = (nq + kDQ - 1) / kDQ, n_tiles = ix.n_tiles * (kTileE / kDE);
    const int64_t cap = map_cap(ix.ws);
    if (onepass) {
        int64_t tpc = 0, chunks = 0;
        const int64_t per = std::max<int64_t>(1, cap / onepass_tile_words(ix, n_qt, &tpc, &chunks));
        return 3 * ((n_qt + per - 1) / per);
    }
    int64_t launches = 0;
    for (int64_t qt0 = 0; qt0 < n_qt;) {
        const int64_t nqt = phase2_pass_tiles(n_tiles, n_qt, qt0, num_sms(), ix.units_per_cta, cap);
        if (nqt == 0) break;
        launches += 2;
        qt0 += nqt;
    }
    return launches;
}

template <int KP, bool F8>
static cudaError_t launch_extract(const ExtractParams &x, bool codes, cudaStream_t st) {
    if (x.chunks > 65535) return cudaErrorInvalidConfiguration;
    const dim3 grid((unsigned)(x.q_pad / 256), (unsigned)x.chunks);
    if (codes)
        k_dense_extract_codes<KP, F8><<<grid, 256, 0, st>>>(x);
    else
        k_dense_extract<KP, F8><<<grid, 256, 0, st>>>(x);
    return cudaGetLastError();
}

static cudaError_t launch_extract_any(int kp, bool f8, const ExtractParams &x, bool codes, cudaStream_t st) {
    switch (kp) {
        case 16: return f8 ? launch_extract<16, true>(x, codes, st) : launch_extract<16, false>(x, codes, st);
        case 32: return f8 ? launch_extract<32, true>(x, codes, st) : launch_extract<32, false>(x, codes, st);
        case 64: return f8 ? launch_extract<64, true>(x, codes, st) : launch_extract<64, false>(x, codes, st);
    }
    return cudaErrorNotSupported;
}

// Fields shared by every dense launch of index ix (PHASE-specific fields left zero).
static DenseParams dense_base(const Index &ix) {
    const Workspace &ws = ix.ws;
    const bool f8 = ix.prefix == HN_PREFIX_FP8_E4M3;
    DenseParams p{};
    // the BF16 prefix, or the FP8 tiles; the queries' BF16 A tiles, or their hi/lo e4m3 bytes
    p.g.pre = f8 ? (const void *)ix.pre8 : (const void *)ix.pre16;
    p.g.qpre = (const void *)ws.qpre16;
    p.g.n = ix.n;
    p.g.n_tiles = ix.n_tiles * (kTileE / kDE);  // index rows are padded to 256: whole 128-entry tiles
    p.status = ws.status;
    p.wait_ns = ws.wait_ns ? ws.wait_ns : kWaitLimitNs;
    p.stall = ws.stall;
    p.plain = ws.plain;
    p.g.code_inv = ix.code_inv;
    p.code_base = code_base();
    return p;
}

static ExtractParams extract_base(const Index &ix, int64_t q0, int64_t nq_pass, int64_t nqt) {
    const Workspace &ws = ix.ws;
    ExtractParams x{};
    x.pre = ix.prefix == HN_PREFIX_FP8_E4M3 ? (const void *)ix.pre8 : (const void *)ix.pre16;
    x.qpre32 = ws.qpre32 + q0 * ix.k_pad4;
    x.gbits = ws.gbits;
    x.n = ix.n;
    x.n_tiles = ix.n_tiles * (kTileE / kDE);
    x.nq = nq_pass;
    x.q_pad = nqt * kDQ;
    x.tau = ws.tau + q0;
    x.bucket = ws.bucket + q0 * ws.bucket_cap;
    x.count = ws.count + q0;
    x.cap = ws.bucket_cap;
    x.code_inv = ix.code_inv;
    x.code_base = code_base();
    x.counters = ws.counters;
    return x;
}

cudaError_t launch_dense_scan(const Index &ix, int64_t nq, int phase, cudaStream_t st) {
    if (!dense_scan_supported(ix)) return cudaErrorNotSupported;
    const Workspace &ws = ix.ws;
    DenseParams p = dense_base(ix);
    const int G = num_sms();
    const int64_t n_qt = (nq + kDQ - 1) / kDQ;
    const int kp = ix.k_pad16;
    const bool f8 = ix.prefix == HN_PREFIX_FP8_E4M3;
    if (phase == 1) {
        // Algorithm 1's Phase 1: the one-pass scan's epilogue without its code map -- the
        // best 32-entry group per (query, entry chunk, tile parity) from the reducing loads
        int64_t tpc = 0, chunks = 0;
        onepass_tile_words(ix, n_qt, &tpc, &chunks);
        DenseParams p4 = dense_base(ix);
        p4.g.nq = nq;
        p4.g.n_qt = n_qt;
        p4.g.tiles_per_chunk = tpc;
        p4.g.chunks = chunks;
        p4.g.words = tpc;
        p4.g.gbits = ws.gbits;
        p4.g.cand = ws.cand;
        p4.n_units = n_qt * chunks;
        if (!onepass_chunking_ok(p4.g) || 2 * chunks > ws.cand_slots) return cudaErrorInvalidValue;
        return launch_dense_kernel(kp, f8, p4, 1, (int)min64(G, p4.n_units), st);
    }
    // Phase 2: the tensor-core scan marks the passing 32-entry groups, k_dense_extract turns
    // them into survivors; passes over query tiles keep the bitmap within the workspace
    const int64_t cap = map_cap(ws);
    for (int64_t qt0 = 0; qt0 < n_qt;) {
        const int64_t nqt = phase2_pass_tiles(p.g.n_tiles, n_qt, qt0, G, ix.units_per_cta, cap);
        if (nqt == 0) return cudaErrorInvalidValue;  // prepare_search sizes the bitmap for one tile at least
        const int64_t q0 = qt0 * kDQ;
        qt0 += nqt;
        DenseParams pp = p;
        int64_t chunks = 0;
        pp.g.qpre = static_cast<const char *>(p.g.qpre) + q0 * kp * 2;  // 2 kp bytes a query (BF16, or e4m3 hi + lo)
        pp.g.nq = min64(nq - q0, nqt * kDQ);
        pp.g.n_qt = nqt;
        dense_chunking(p.g.n_tiles, nqt, G, ix.units_per_cta, &pp.g.tiles_per_chunk, &chunks);
        pp.g.chunks = chunks;
        pp.n_units = nqt * chunks;
        pp.g.tau = ws.tau + q0;
        pp.g.gbits = ws.gbits;
        pp.g.words = (pp.g.tiles_per_chunk + 15) / 16;
        ExtractParams x = extract_base(ix, q0, pp.g.nq, nqt);
        x.tiles_per_chunk = pp.g.tiles_per_chunk;
        x.chunks = chunks;
        x.words = pp.g.words;
        cudaError_t e = launch_dense_kernel(kp, f8, pp, 2, (int)min64(G, pp.n_units), st);
        if (e == cudaSuccess) e = launch_extract_any(kp, f8, x, false, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One-pass dense search steps, per pass over query tiles: the PHASE-4 scan (group codes and
// threshold candidates), the threshold from the candidates, and the code-map extraction.
// With `ev` (3 events), the first pass records ev[0] after its scan, ev[1] after its
// threshold and ev[2] after the last pass's extraction.
cudaError_t launch_dense_onepass(const Index &ix, const float *q, int64_t nq, int kk, bool keep_best,
                                 cudaStream_t st, cudaEvent_t *ev) {
    if (!dense_scan_supported(ix)) return cudaErrorNotSupported;
    const Workspace &ws = ix.ws;
    const int G = num_sms();
    const int64_t n_qt = (nq + kDQ - 1) / kDQ;
    const int kp = ix.k_pad16;
    const bool f8 = ix.prefix == HN_PREFIX_FP8_E4M3;
    int64_t tpc = 0, chunks = 0;
    const int64_t tile_words = onepass_tile_words(ix, n_qt, &tpc, &chunks);
    const int64_t per = map_cap(ws) / tile_words;  // query tiles per pass
    if (per < 1) return cudaErrorInvalidValue;      // prepare_search sizes the map for one tile at least
    const int S = (int)(2 * chunks);                // candidate slots per query
    if (S > ws.cand_slots) return cudaErrorInvalidValue;
    DenseParams p = dense_base(ix);
    p.g.tiles_per_chunk = tpc;
    p.g.chunks = chunks;
    p.g.words = tpc;
    p.g.gbits = ws.gbits;
    if (!onepass_chunking_ok(p.g)) return cudaErrorInvalidValue;
    for (int64_t qt0 = 0; qt0 < n_qt;) {
        const int64_t nqt = std::min(per, n_qt - qt0);
        const int64_t q0 = qt0 * kDQ;
        const bool first = qt0 == 0;
        qt0 += nqt;
        DenseParams pp = p;
        pp.g.qpre = static_cast<const char *>(p.g.qpre) + q0 * kp * 2;
        pp.g.nq = min64(nq - q0, nqt * kDQ);
        pp.g.n_qt = nqt;
        pp.n_units = nqt * chunks;
        pp.g.cand = ws.cand + q0 * S;
        cudaError_t e = launch_dense_kernel(kp, f8, pp, 4, (int)min64(G, pp.n_units), st);
        if (e == cudaSuccess && ev && first) e = cudaEventRecord(ev[0], st);
        if (e == cudaSuccess) e = launch_seed_threshold_at(ix, q, q0, pp.g.nq, S, 32, kk, keep_best, st);
        if (e == cudaSuccess && ev && first) e = cudaEventRecord(ev[1], st);
        ExtractParams x = extract_base(ix, q0, pp.g.nq, nqt);
        x.tiles_per_chunk = tpc;
        x.chunks = chunks;
        x.words = pp.g.words;
        if (e == cudaSuccess) e = launch_extract_any(kp, f8, x, true, st);
        if (e != cudaSuccess) return e;
    }
    return ev ? cudaEventRecord(ev[2], st) : cudaSuccess;
}

// Verification: every prefix score of nq prepared queries (ws.qpre*) against the index,
// [nq][n] FP32, from the tensor-core scan's Phase-2 arithmetic (path 0) or the CUDA-core
// FMA chain of the survivor extraction (path 1).
cudaError_t launch_prefix_scores(const Index &ix, int64_t nq, int path, float *out, cudaStream_t st) {
    if (!dense_scan_supported(ix)) return cudaErrorNotSupported;
    const int kp = ix.k_pad16;
    const bool f8 = ix.prefix == HN_PREFIX_FP8_E4M3;
    if (path == 0) {
        DenseParams p = dense_base(ix);
        int64_t chunks = 0;
        p.g.nq = nq;
        p.g.n_qt = (nq + kDQ - 1) / kDQ;
        dense_chunking(p.g.n_tiles, p.g.n_qt, num_sms(), ix.units_per_cta, &p.g.tiles_per_chunk, &chunks);
        p.g.chunks = chunks;
        p.n_units = p.g.n_qt * chunks;
        p.dump = out;
        return launch_dense_kernel(kp, f8, p, 3, (int)min64(num_sms(), p.n_units), st);
    }
    ExtractParams x = extract_base(ix, 0, nq, (nq + kDQ - 1) / kDQ);
    const int64_t total = nq * ix.n;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    switch (kp) {
        case 16: f8 ? k_fma_scores<16, true><<<blocks, 256, 0, st>>>(x, out) : k_fma_scores<16, false><<<blocks, 256, 0, st>>>(x, out); break;
        case 32: f8 ? k_fma_scores<32, true><<<blocks, 256, 0, st>>>(x, out) : k_fma_scores<32, false><<<blocks, 256, 0, st>>>(x, out); break;
        case 64: f8 ? k_fma_scores<64, true><<<blocks, 256, 0, st>>>(x, out) : k_fma_scores<64, false><<<blocks, 256, 0, st>>>(x, out); break;
        default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace hn

namespace hn {

// ------------------------------------------------------------------ batched serving
// One persistent one-pass scan over several groups (an index and its concatenated
// queries each).  Every joined group keeps its own code map, candidate slots and
// threshold; only the scan is shared, so that small groups fill the SMs together
// instead of one full-GPU launch each.  A group joins when its index has the common
// tile format and its code map holds the whole group in one pass.
struct DenseMulti {
    std::vector<const Index *> ix;
    std::vector<DenseGroup> g;          // host copy of the descriptors
    DenseGroup *dev = nullptr;          // device copy
    int64_t n_units = 0;
    int kp = 16;
    bool f8 = false;
};


bool dense_multi_joinable(const Index &ix, int64_t nq, int kp, bool f8) {
    if (!dense_scan_supported(ix) || ix.k_pad16 != kp || (ix.prefix == HN_PREFIX_FP8_E4M3) != f8 || nq < 1) return false;
    int64_t tpc = 0, chunks = 0;
    multi_chunking(ix, nq, &tpc, &chunks);
    const int64_t n_qt = (nq + kDQ - 1) / kDQ;
    return 2 * chunks <= ix.ws.cand_slots && chunks * tpc * n_qt * kDQ <= ix.ws.gbits_cap;
}

hn_status dense_multi_create(const std::vector<const Index *> &ixs, const std::vector<int64_t> &nqs,
                             DenseMulti **out) {
    *out = nullptr;
    if (ixs.empty() || ixs.size() != nqs.size()) return fail(HN_ERR_INVALID_ARG, "dense_multi_create: no groups");
    DenseMulti *m = new DenseMulti();
    m->kp = ixs[0]->k_pad16;
    m->f8 = ixs[0]->prefix == HN_PREFIX_FP8_E4M3;
    for (size_t i = 0; i < ixs.size(); ++i) {
        const Index &ix = *ixs[i];
        if (!dense_multi_joinable(ix, nqs[i], m->kp, m->f8)) {
            delete m;
            return fail(HN_ERR_INVALID_ARG, "dense_multi_create: a group cannot join");
        }
        DenseGroup g{};
        g.pre = m->f8 ? (const void *)ix.pre8 : (const void *)ix.pre16;
        g.qpre = ix.ws.qpre16;
        g.n = ix.n;
        g.n_tiles = ix.n_tiles * (kTileE / kDE);
        g.nq = nqs[i];
        g.n_qt = (nqs[i] + kDQ - 1) / kDQ;
        multi_chunking(ix, nqs[i], &g.tiles_per_chunk, &g.chunks);
        g.unit0 = m->n_units;
        g.cand = ix.ws.cand;
        g.gbits = ix.ws.gbits;
        g.words = g.tiles_per_chunk;
        g.code_inv = ix.code_inv;
        if (!onepass_chunking_ok(g)) {
            delete m;
            return fail(HN_ERR_UNSUPPORTED, "dense_multi_create: odd chunking");
        }
        m->n_units += g.n_qt * g.chunks;
        m->ix.push_back(&ix);
        m->g.push_back(g);
    }
    cudaError_t e = cudaMalloc(&m->dev, sizeof(DenseGroup) * m->g.size());
    if (e == cudaSuccess) e = cudaMemcpy(m->dev, m->g.data(), sizeof(DenseGroup) * m->g.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        delete m;
        return cuda_fail(e, "dense_multi_create");
    }
    *out = m;
    return HN_OK;
}

void dense_multi_destroy(DenseMulti *m) {
    if (!m) return;
    cudaFree(m->dev);
    delete m;
}

template <int KP, bool F8>
static cudaError_t launch_multi_kp(const DenseParams &p, int grid, cudaStream_t st) {
    if (reg_split_ok<KP, 4, F8, true>())
        k_dense_scan<KP, 4, F8, true, true><<<grid, kDenseThreads, dense_smem<KP, 4, F8>(), st>>>(p);
    else
        k_dense_scan<KP, 4, F8, true><<<grid, kDenseThreads, dense_smem<KP, 4, F8>(), st>>>(p);
    return cudaGetLastError();
}

cudaError_t dense_multi_scan(const DenseMulti *m, cudaStream_t st) {
    cudaError_t e = dense_init();
    if (e != cudaSuccess) return e;
    DenseParams p{};
    p.groups = m->dev;
    p.n_groups = (int32_t)m->g.size();
    p.n_units = m->n_units;
    p.code_base = code_base();
    p.wait_ns = kWaitLimitNs;
    p.status = m->ix[0]->ws.status;   // a timeout is reported through the first group's status word
    const int grid = (int)min64(num_sms(), m->n_units);
    switch (m->kp) {
        case 16: return m->f8 ? launch_multi_kp<16, true>(p, grid, st) : launch_multi_kp<16, false>(p, grid, st);
        case 32: return m->f8 ? launch_multi_kp<32, true>(p, grid, st) : launch_multi_kp<32, false>(p, grid, st);
        case 64: return m->f8 ? launch_multi_kp<64, true>(p, grid, st) : launch_multi_kp<64, false>(p, grid, st);
    }
    return cudaErrorNotSupported;
}

// Group gi after the shared scan: the threshold from its candidates, then its survivors
// from its code map (queries q, HN-normalised, as prepared).
cudaError_t dense_multi_post(const DenseMulti *m, int gi, const float *q, cudaStream_t st) {
    const Index &ix = *m->ix[gi];
    const DenseGroup &g = m->g[gi];
    cudaError_t e = launch_seed_threshold_at(ix, q, 0, g.nq, (int)(2 * g.chunks), 32, 1, false, st);
    if (e != cudaSuccess) return e;
    ExtractParams x = extract_base(ix, 0, g.nq, g.n_qt);
    x.tiles_per_chunk = g.tiles_per_chunk;
    x.chunks = g.chunks;
    x.words = g.words;
    return launch_extract_any(m->kp, m->f8, x, true, st);
}

}  // namespace hn
