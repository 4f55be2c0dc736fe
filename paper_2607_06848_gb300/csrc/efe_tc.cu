// Cell products Y_e = H_e X'_e on the 5th-generation tensor cores (tcgen05,
// sm_103a): bf16 operands, FP32 accumulation in tensor memory.
//
// Layout choices (all produced by this library, so chosen for the MMA):
//   A = H_e (ne x ne, bf16) is stored per cell pre-tiled in the canonical
//       K-major no-swizzle layout, k-step by k-step: for k-step s (16
//       columns) and M-tile mt (128 rows) a 4 KB block of 8x8 core matrices,
//       core (rg, kg) at byte (rg*2 + kg)*128, blocks ordered [s][mt].  One
//       A stage (all M-tiles of one k-step) is a single 1-D bulk copy
//       (LBO = 128 B along K, SBO = 256 B along M).
//   B = X'_e (K x Npad, bf16) is gathered by TMA straight from the node grid:
//       a 4-D tile {8 columns, xpad, p+1, 1} per z-plane and column block
//       lands as rows of 16 B, i.e. the canonical MN-major no-swizzle layout.
//       Planes are grouped in pairs; a pair is 2 (p+1) xpad rows = (p+1)
//       whole k-steps, held in one of two ring slots (LBO = 128 B between
//       8-row K groups, SBO = 2 (p+1) xpad 16 B between 8-column blocks).  No
//       index list: the cell's nodes are a box.  The x extent is padded to
//       xpad = 8 so that every plane is a multiple of 128 B (TMA destinations
//       must be 128-byte aligned); the padding node meets zero columns of the
//       pre-tiled H_e.  K index k = (z*(p+1) + y)*xpad + x.
//   D = accumulator, M-tile mt at TMEM columns [mt*Npad, (mt+1)*Npad).
// The MMAs run k-step-major (all M-tiles of a k-step, then the next k-step),
// so each plane pair is released as soon as its k-steps are done and the
// freed shared memory deepens the A ring.  An A stage holds several k-steps
// (one bulk copy and one barrier round trip per stage: the round trip, not the
// data, bounds a stage of a single k-step).  Each tcgen05.mma costs about the
// same issue time whatever its N, so all columns go into one instruction
// (N up to 512 / MT) and the accumulators fill most of the SM's tensor memory;
// when two buffers fit (small N) the epilogue of one cell overlaps the MMAs of
// the next, otherwise the MMAs wait for it, and twelve epilogue warps (three
// per TMEM lane quadrant) keep that drain short.  Columns beyond one
// instruction's N go to further chunks, one per block of a thread-block
// cluster; the cluster's blocks walk the same cells, and its first block
// loads each A stage (H_e tiles, coupling tiles) once and multicasts it to
// all of them, whose MMAs each release the stage (a multicast commit to the
// empty barriers of every block).
// Coupling (the bf16 filter): the FE rows of H^E Y also hold E^T Y_e + P_c^T W
// (the FE-enrichment block of H^E and the projector rows).  Each FE node is
// owned by exactly one cell (the one in which its local indices lie in
// [0, p)^3), and a cell's owned rows receive these terms as extra k-steps of
// the same accumulation: A holds, per extra k-step, the coefficients of two
// atoms (8 columns each: E_f, P_c,f for f = s, px, py, pz; zero for rows the
// cell does not own), B the rows Y_e(atom) and W(atom) (8 rows per atom,
// one bulk copy per atom from a table laid out as MN-major core matrices).
// So the coupling runs on the tensor cores, and the node kernel that sums the
// cells is a plain streaming pass.
// E Y_c of the enriched rows rides in the padding rows of the last M-tile
// (rows n_e .. MT*128 of A hold the cell's E coefficients, four per
// cell-atom pair): their accumulators go to FP32 partials per pair.
// Per-cell results go to Ycells[cell][row][ldy] (FP32 or bf16); a gather
// kernel sums the up-to-8 contributions of each node, so no colouring or
// atomics are needed and every cell of the mesh runs in one persistent launch.
// The epilogue reads each thread's row (TMEM lane) in 16-column groups.  bf16
// rows whose stride is a whole number of 32-byte spans are staged in shared
// memory as 32-row x 16-column boxes (32-byte swizzle) and leave by TMA tensor
// stores, so the accumulator is released without waiting for global stores;
// other rows are stored directly, in whole 32-byte sectors.
#include "efe_internal.cuh"
#include <cstring>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>

namespace {

constexpr int EPI_WARPS = 12;        // epilogue: three warps per TMEM lane quadrant, splitting the columns
constexpr int TC_THREADS = 128 + 32 * EPI_WARPS;   // w0 TMA producer, w1 MMA issuer, w2 TMEM owner, w4.. epilogue
constexpr int MAX_A_STAGES = 24;     // A ring depth limit (one stage = one k-step of all M-tiles)
constexpr int B_SLOTS = 2;           // plane-pair ring
constexpr int SMEM_LIMIT = 232448;   // dynamic shared memory per block (227 KB, one block per SM)
constexpr int TMEM_COLS = 512;       // tensor memory per block: one or two accumulator buffers
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz before a wait gives up
constexpr int EPI_SLOT = 1024;       // epilogue staging: one 32-row x 16-column bf16 box (32-byte rows)
constexpr int EPI_STAGE = EPI_WARPS * 2 * EPI_SLOT;   // two slots per epilogue warp

struct TcParams {
    int ncells, nx, ny, p, np1, ne, xpad, Kpad, ksteps, MT, Npad, ncb, ldy;   // column chunk: blockIdx.y
    int plane_rows;                     // (p+1) xpad rows per z-plane
    int kpg;                            // k-steps per plane pair: 2 plane_rows / 16
    int ngroups;                        // plane pairs per cell: ceil((p+1) / 2)
    int a_stages;                       // A ring depth
    int ks;                             // k-steps per A stage (one bulk copy, one barrier pair)
    int slot_bytes;                     // one B slot: ncb x 2 plane_rows x 16 B
    int out_bf16;                       // per-cell results stored as bf16 (else FP32)
    // coupling as extra k-steps (cx_off == nullptr: none)
    const int *cx_off;                  // ncells + 1: first extra k-step of each cell
    const int *cx_atoms;                // 2 atom slots per extra k-step (natoms: the zero block)
    const __nv_bfloat16 *Ax;            // extra A stages [k-step][MT][2048]
    const __nv_bfloat16 *YW;            // [atom][nCB][8 rows][8 columns]: Y_e (rows 0-3), W (rows 4-7)
    int ncl;                            // blocks per cluster = column chunks (blockIdx.y)
    int nbuf;                           // accumulator buffers in tensor memory (1 or 2)
    int nCB;                            // 8-column blocks per atom in YW
    int x_slot_bytes;                   // shared memory of the extra B slot
    float *Epart;                       // E Y_c per (cell-atom pair, f) from the padding rows (nullptr: none)
    const int *ca_ptr;                  // ncells + 1: the cell-atom pairs of each cell
    int tma_out;                        // bf16 rows leave by TMA tensor stores (ymap valid)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false after ~WAIT_CYCLES (the caller records the error and stops).
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity) {
    if (mbar_try(b, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try(b, parity)) {
        if (clock64() - t0 > WAIT_CYCLES) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// the same, delivered to the same shared-memory offset in every block of the
// cluster in `mask`, signalling the barrier at that offset in each of them
__device__ __forceinline__ void bulk_load_mc(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                             uint16_t mask) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar)), "h"(mask)
        : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared-memory matrix descriptor, no swizzle (layout type 0), version 1
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// commit that arrives on the barrier at this offset in every block of `mask`
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// TMEM -> registers, 16 consecutive columns of the warp's 32 lanes (rows)
// (no wait: several are issued, then one tmem_wait_ld())
__device__ __forceinline__ void tmem_ld16_nw(uint32_t taddr, uint32_t r[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// ties the registers of a load to a point after tmem_wait_ld(), so that no use
// of them is scheduled before the wait
__device__ __forceinline__ void reg_after_wait(uint32_t r[16]) {
    asm volatile(""
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]));
}

// shared -> global through the tensor map (bf16 output rows): box {16 columns,
// 32 rows, 1 cell} at (x, y, z); rows past n_e and columns past ldy lie outside
// the map and are not written.  Completion is tracked per thread in bulk groups.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_le1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ uint32_t pack_bf16(uint32_t lo, uint32_t hi) {
    __nv_bfloat162 b2 = __floats2bfloat162_rn(__uint_as_float(lo), __uint_as_float(hi));
    return *reinterpret_cast<uint32_t *>(&b2);
}

// Columns col .. col+15 of one output row from 16 FP32 accumulators: bf16 (32
// bytes) or FP32 (64 bytes); 256-bit stores when `wide` (aligned), else 16-byte
// stores; nothing at or past ldy (ldy is a multiple of 8 for bf16, of 4 for FP32).
__device__ __forceinline__ void store16(unsigned char *row, int col, int ldy, int bf16, bool wide,
                                        const uint32_t v[16]) {
    if (bf16) {
        uint32_t w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            __nv_bfloat162 b2 = __floats2bfloat162_rn(__uint_as_float(v[2 * i]), __uint_as_float(v[2 * i + 1]));
            w[i] = *reinterpret_cast<uint32_t *>(&b2);
        }
        unsigned char *p = row + (size_t)col * 2;
        if (wide && col + 16 <= ldy) {
            asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                         "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                         : "memory");
        } else {
            if (col + 8 <= ldy) *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
            if (col + 16 <= ldy) *reinterpret_cast<uint4 *>(p + 16) = make_uint4(w[4], w[5], w[6], w[7]);
        }
    } else {
        unsigned char *p = row + (size_t)col * 4;
        if (wide && col + 16 <= ldy) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p + 32 * h),
                             "r"(v[8 * h]), "r"(v[8 * h + 1]), "r"(v[8 * h + 2]), "r"(v[8 * h + 3]), "r"(v[8 * h + 4]),
                             "r"(v[8 * h + 5]), "r"(v[8 * h + 6]), "r"(v[8 * h + 7])
                             : "memory");
        } else {
#pragma unroll
            for (int h = 0; h < 4; ++h)
                if (col + 4 * h + 4 <= ldy)
                    *reinterpret_cast<uint4 *>(p + 16 * h) = make_uint4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        }
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_cell_mma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
               const __nv_bfloat16 *__restrict__ He16, void *Ycells, TcParams P, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // every TMA destination below is a multiple of 128 B from this base
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int stage_bytes = P.ks * P.MT * 4096;      // one A stage: ks k-steps of all M-tiles
    unsigned char *sE = smem;                          // epilogue staging (bf16 output boxes)
    unsigned char *sA = smem + EPI_STAGE;
    unsigned char *sB = sA + (size_t)P.a_stages * stage_bytes;
    unsigned char *sX = sB + (size_t)B_SLOTS * P.slot_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sX + P.x_slot_bytes);
    uint64_t *full_a = bars, *empty_a = bars + MAX_A_STAGES;
    uint64_t *full_b = bars + 2 * MAX_A_STAGES, *empty_b = full_b + B_SLOTS;
    uint64_t *acc_full = empty_b + B_SLOTS, *acc_empty = acc_full + 8;   // [buffer][M-tile]
    uint64_t *full_x = acc_empty + 8, *empty_x = full_x + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty_x + 1);
    const uint32_t xblk = (uint32_t)P.ncb * 128;      // one atom's 8 rows x Npad columns in sX

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair_stride = 2 * P.plane_rows * 16;   // bytes between column blocks in a slot
    const int col0 = blockIdx.y * P.Npad;             // this block's column chunk (its rank in the cluster)
    const bool leader = blockIdx.y == 0;               // loads (and multicasts) the A stages
    const uint16_t cmask = (uint16_t)((1u << P.ncl) - 1u);
    const uint32_t acc_cols = (uint32_t)(P.MT * P.Npad);   // one accumulator buffer

    if (threadIdx.x == 0) {
        // an A stage is released by the MMAs of every block of the cluster
        for (int i = 0; i < P.a_stages; ++i) { mbar_init(&full_a[i], 1); mbar_init(&empty_a[i], P.ncl); }
        for (int i = 0; i < B_SLOTS; ++i) { mbar_init(&full_b[i], 1); mbar_init(&empty_b[i], 1); }
        for (int t = 0; t < 8; ++t) { mbar_init(&acc_full[t], 1); mbar_init(&acc_empty[t], 32 * EPI_WARPS); }
        mbar_init(full_x, 1);
        mbar_init(empty_x, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero both B slots once: rows a lone last plane leaves unwritten meet zero
    // columns of H_e, and must hold finite values
    for (int i = threadIdx.x; i < (B_SLOTS * P.slot_bytes + P.x_slot_bytes) / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(sB)[i] = 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        fence_before();
    }
    __syncthreads();
    fence_after();
    // every block's barriers exist before any multicast or remote arrive reaches them
    cluster_sync_all();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        // A stages of up to KS k-steps (one bulk copy each, multicast by the
        // leader); before a stage, the plane pairs its k-steps read
        int sa = 0, sb = 0;
        uint32_t pha = 0, phb = 0;
        bool ok = true;
        uint32_t aused = 0, apar = 0;      // per A slot: issued at least once, parity of its last phase
        uint32_t bused = 0, bpar = 0;      // the same per B slot
        uint32_t phx = 0, xused = 0, xpar = 0;
        auto load_a = [&](const __nv_bfloat16 *src, int cnt) -> bool {
            if (!mbar_wait(&empty_a[sa], pha ^ 1)) return false;
            const uint32_t bytes = (uint32_t)(cnt * P.MT * 4096);
            mbar_expect_tx(&full_a[sa], bytes);
            if (P.ncl == 1) bulk_load(sA + (size_t)sa * stage_bytes, src, bytes, &full_a[sa]);
            else if (leader) bulk_load_mc(sA + (size_t)sa * stage_bytes, src, bytes, &full_a[sa], cmask);
            aused |= 1u << sa;
            apar = (apar & ~(1u << sa)) | (pha << sa);
            if (++sa == P.a_stages) { sa = 0; pha ^= 1; }
            return true;
        };
        for (int cell = blockIdx.x; cell < P.ncells && ok; cell += gridDim.x) {
            const int cx = cell % P.nx, cy = (cell / P.nx) % P.ny, cz = cell / (P.nx * P.ny);
            const __nv_bfloat16 *Ac = He16 + (size_t)cell * P.ksteps * P.MT * 2048;
            int gnext = 0;
            for (int s = 0; s < P.ksteps && ok; s += P.ks) {
                const int cnt = min(P.ks, P.ksteps - s);
                // plane pairs read by k-steps < s + cnt
                while (ok && gnext < P.ngroups && gnext * P.kpg < s + cnt) {
                    const int g = gnext++;
                    if (!mbar_wait(&empty_b[sb], phb ^ 1)) { ok = false; break; }
                    const int np = min(2, P.np1 - 2 * g);
                    mbar_expect_tx(&full_b[sb], (uint32_t)(np * P.plane_rows * 16 * P.ncb));
                    unsigned char *slot = sB + (size_t)sb * P.slot_bytes;
                    for (int zz = 0; zz < np; ++zz)
                        for (int cb = 0; cb < P.ncb; ++cb)
                            tma_load_4d(slot + (size_t)cb * pair_stride + (size_t)zz * P.plane_rows * 16, &xmap,
                                        col0 + 8 * cb, cx * P.p, cy * P.p, cz * P.p + 2 * g + zz,
                                        &full_b[sb]);   // {cols, x, y, z}
                    bused |= 1u << sb;
                    bpar = (bpar & ~(1u << sb)) | (phb << sb);
                    if (++sb == B_SLOTS) { sb = 0; phb ^= 1; }
                }
                if (!ok || !load_a(Ac + (size_t)s * P.MT * 2048, cnt)) { ok = false; break; }
            }
            // the coupling: Y_e / W rows of the cell's atoms, then its extra A stages
            const int x0 = P.cx_off ? P.cx_off[cell] : 0;
            const int nxs = P.cx_off ? P.cx_off[cell + 1] - x0 : 0;
            if (ok && nxs > 0) {
                if (!mbar_wait(empty_x, phx ^ 1)) { ok = false; break; }
                mbar_expect_tx(full_x, (uint32_t)(2 * nxs) * xblk);
                for (int sl = 0; sl < 2 * nxs; ++sl) {
                    const int atom = P.cx_atoms[2 * x0 + sl];
                    bulk_load(sX + (size_t)sl * xblk, P.YW + ((size_t)atom * P.nCB + col0 / 8) * 64, xblk, full_x);
                }
                xused = 1;
                xpar = phx;
                phx ^= 1;
                for (int j = 0; j < nxs && ok; j += P.ks)
                    if (!load_a(P.Ax + (size_t)(x0 + j) * P.MT * 2048, min(P.ks, nxs - j))) ok = false;
            }
        }
        if (!ok) atomicExch(err, 1);
        if (xused) mbar_wait(full_x, xpar);
        // drain: every copy this thread issued (or expects) has landed before the block exits
        for (int i = 0; i < B_SLOTS; ++i)
            if (bused & (1u << i)) mbar_wait(&full_b[i], (bpar >> i) & 1u);
        for (int i = 0; i < P.a_stages; ++i)
            if (aused & (1u << i)) mbar_wait(&full_a[i], (apar >> i) & 1u);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                               ((uint32_t)(P.Npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        int sa = 0, sb = 0;
        uint32_t pha = 0, phb = 0, phx = 0;
        int it = 0;
        bool ok = true;
        const uint32_t sB_addr = smem_u32(sB), sA_addr = smem_u32(sA), sX_addr = smem_u32(sX);
        // descriptors differ only in the 14-bit start-address field (shared
        // addresses < 256 KB): a base descriptor plus (byte offset >> 4)
        const uint64_t adesc0 = smem_desc(sA_addr, 128, 256);
        const uint64_t bdesc0 = smem_desc(sB_addr, 128, (uint32_t)pair_stride);
        for (int cell = blockIdx.x; cell < P.ncells && ok; cell += gridDim.x, ++it) {
            // accumulator buffer of this cell: every M-tile of it must be drained
            const int buf = it % P.nbuf, use = it / P.nbuf;
            const uint32_t dacc = tmem + (uint32_t)buf * acc_cols;
            for (int mt = 0; mt < P.MT && ok; ++mt)
                if (!mbar_wait(&acc_empty[4 * buf + mt], (use & 1) ^ 1)) ok = false;
            if (!ok) break;
            fence_after();
            int j = 0;                                        // k-step within the current plane pair
            for (int s0 = 0; s0 < P.ksteps && ok; s0 += P.ks) {
                const int cnt = min(P.ks, P.ksteps - s0);
                if (!mbar_wait(&full_a[sa], pha)) { ok = false; break; }
                fence_after();
                uint64_t ad = adesc0 + (uint64_t)(((uint32_t)sa * (uint32_t)stage_bytes) >> 4);
                for (int t = 0; t < cnt; ++t, ad += (uint64_t)(P.MT * 4096 >> 4)) {
                    const int s = s0 + t;
                    if (j == 0) {
                        if (!mbar_wait(&full_b[sb], phb)) { ok = false; break; }
                        fence_after();
                    }
                    const uint64_t bd = bdesc0 + (uint64_t)(((uint32_t)sb * (uint32_t)P.slot_bytes + j * 256) >> 4);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    for (int mt = 0; mt < P.MT; ++mt)
                        mma_bf16(dacc + (uint32_t)(mt * P.Npad), ad + (uint64_t)(mt * 256), bd, idesc, acc);
                    if (++j == P.kpg || s == P.ksteps - 1) {
                        mma_commit(&empty_b[sb]);
                        if (++sb == B_SLOTS) { sb = 0; phb ^= 1; }
                        j = 0;
                    }
                }
                if (!ok) break;
                if (P.ncl == 1) mma_commit(&empty_a[sa]);
                else mma_commit_mc(&empty_a[sa], cmask);
                if (++sa == P.a_stages) { sa = 0; pha ^= 1; }
            }
            if (!ok) break;
            const int x0 = P.cx_off ? P.cx_off[cell] : 0;
            const int nxs = P.cx_off ? P.cx_off[cell + 1] - x0 : 0;
            if (nxs > 0) {
                if (!mbar_wait(full_x, phx)) { ok = false; break; }
                fence_after();
                for (int j0 = 0; j0 < nxs && ok; j0 += P.ks) {
                    const int cnt = min(P.ks, nxs - j0);
                    if (!mbar_wait(&full_a[sa], pha)) { ok = false; break; }
                    fence_after();
                    for (int t = 0; t < cnt; ++t) {
                        // two atoms (16 K rows): K groups xblk apart, 8-column blocks 128 B apart
                        const uint64_t bd = smem_desc(sX_addr + (uint32_t)(2 * (j0 + t)) * xblk, xblk, 128);
                        const uint32_t abase = sA_addr + sa * stage_bytes + t * P.MT * 4096;
                        for (int mt = 0; mt < P.MT; ++mt)
                            mma_bf16(dacc + (uint32_t)(mt * P.Npad), smem_desc(abase + mt * 4096, 128, 256), bd,
                                     idesc, 1u);
                    }
                    if (P.ncl == 1) mma_commit(&empty_a[sa]);
                    else mma_commit_mc(&empty_a[sa], cmask);
                    if (++sa == P.a_stages) { sa = 0; pha ^= 1; }
                }
                if (!ok) break;
                mma_commit(empty_x);
                phx ^= 1;
            }
            for (int mt = 0; mt < P.MT; ++mt) mma_commit(&acc_full[4 * buf + mt]);
        }
        if (!ok) atomicExch(err, 2);
    } else if (warp >= 4) {
        // ---------------- epilogue ----------------
        // TMEM -> registers (thread = row), 64-column chunks, one per warp of
        // the lane quadrant in turn.  bf16 output: the chunk is packed in
        // registers, the accumulator is released, and the rows leave through
        // shared memory by TMA tensor stores (32 rows x 16 columns per box, two
        // staging slots per warp), so the MMAs of the next cell do not wait for
        // the global stores.  FP32 output: direct stores, then the release.
        const int q = warp & 3, ew = (warp - 4) >> 2;   // lane quadrant; which third of the column chunks
        const int eb = P.out_bf16 ? 2 : 4;              // bytes per stored element
        // 32-byte stores need 32-byte aligned rows and chunk starts
        const bool wide = ((size_t)P.ldy * eb) % 32 == 0 && (col0 * eb) % 32 == 0 &&
                          (reinterpret_cast<uintptr_t>(Ycells) & 31) == 0;
        const uint32_t stg = smem_u32(sE + (size_t)(warp - 4) * 2 * EPI_SLOT);
        const bool tma_out = P.tma_out != 0;
        int nst = 0;                                    // boxes this warp has stored (lane 0 issues)
        int it = 0;
        bool ok = true;
        for (int cell = blockIdx.x; cell < P.ncells && ok; cell += gridDim.x, ++it) {
            const int buf = it % P.nbuf, use = it / P.nbuf;
            for (int mt = 0; mt < P.MT; ++mt) {
                // warp-uniform decision: the TMEM loads below are .sync.aligned
                const bool got = mbar_wait(&acc_full[4 * buf + mt], use & 1);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                fence_after();
                const int rbase = mt * 128 + q * 32;
                const uint32_t tbase =
                    tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * acc_cols + (uint32_t)(mt * P.Npad);
                // the padding rows of the last tile carry E Y_c partials (row ne + 4 slot + f)
                auto epart = [&]() {
                    if (!(P.Epart && ew == 0 && mt == P.MT - 1 && rbase + 32 > P.ne)) return;
                    const int q0 = P.ca_ptr[cell];
                    const int nrow = 4 * (P.ca_ptr[cell + 1] - q0);
                    const int r = rbase + lane - P.ne;                 // this lane's padding row
                    float *dst = P.Epart + ((size_t)q0 * 4 + (r > 0 ? r : 0)) * P.ldy + col0;
                    for (int c0 = 0; c0 < P.Npad; c0 += 16) {
                        uint32_t v[16];
                        tmem_ld16_nw(tbase + (uint32_t)c0, v);
                        tmem_wait_ld();
                        reg_after_wait(v);
                        if (r >= 0 && r < nrow) {
#pragma unroll
                            for (int i = 0; i < 16; i += 4)
                                if (col0 + c0 + i < P.ldy)
                                    *reinterpret_cast<float4 *>(dst + c0 + i) =
                                        make_float4(__uint_as_float(v[i]), __uint_as_float(v[i + 1]),
                                                    __uint_as_float(v[i + 2]), __uint_as_float(v[i + 3]));
                        }
                    }
                };
                if (tma_out) {
                    // bf16: 16-column groups -> staging slot -> TMA tensor store (asynchronous,
                    // so the release below does not wait for the global writes)
                    for (int c0 = ew * 64; rbase < P.ne && c0 < P.Npad; c0 += (EPI_WARPS / 4) * 64) {
                        const int nl = min(64, P.Npad - c0) / 16;  // warp-uniform
#pragma unroll
                        for (int g0 = 0; g0 < 4; g0 += 2) {
                            if (g0 >= nl) break;
                            uint32_t r[2][16];
#pragma unroll
                            for (int gg = 0; gg < 2; ++gg)
                                if (g0 + gg < nl) tmem_ld16_nw(tbase + (uint32_t)(c0 + 16 * (g0 + gg)), r[gg]);
                            tmem_wait_ld();
#pragma unroll
                            for (int gg = 0; gg < 2; ++gg) {
                                if (g0 + gg >= nl) continue;
                                reg_after_wait(r[gg]);
                                uint32_t pk[8];
#pragma unroll
                                for (int i = 0; i < 8; ++i) pk[i] = pack_bf16(r[gg][2 * i], r[gg][2 * i + 1]);
                                // 32-byte rows (lane = row), 16-byte halves swapped on rows 4-7 mod 8
                                const uint32_t slot = stg + (uint32_t)(nst & 1) * EPI_SLOT;
                                if (lane == 0 && nst >= 2) bulk_wait_read_le1();   // this slot's last store has read it
                                __syncwarp();
                                const uint32_t sw = (uint32_t)((lane >> 2) & 1);
#pragma unroll
                                for (int h = 0; h < 2; ++h)
                                    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(
                                                     slot + (uint32_t)lane * 32u + ((uint32_t)h ^ sw) * 16u),
                                                 "r"(pk[4 * h]), "r"(pk[4 * h + 1]), "r"(pk[4 * h + 2]),
                                                 "r"(pk[4 * h + 3]));
                                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                                __syncwarp();
                                if (lane == 0) tma_store_3d(&ymap, slot, col0 + c0 + 16 * (g0 + gg), rbase, cell);
                                ++nst;
                            }
                        }
                    }
                    epart();
                    fence_before();
                    mbar_arrive(&acc_empty[4 * buf + mt]);
                } else {
                    // 64-column chunks stored directly, then the release
                    const bool row_ok = rbase + lane < P.ne;
                    unsigned char *yrow = reinterpret_cast<unsigned char *>(Ycells) +
                                          ((size_t)cell * P.ne + rbase + lane) * P.ldy * eb;
                    for (int c0 = ew * 64; rbase < P.ne && c0 < P.Npad; c0 += (EPI_WARPS / 4) * 64) {
                        const int nl = min(64, P.Npad - c0) / 16;  // warp-uniform
                        uint32_t r[4][16];
#pragma unroll
                        for (int g = 0; g < 4; ++g)
                            if (g < nl) tmem_ld16_nw(tbase + (uint32_t)(c0 + 16 * g), r[g]);
                        tmem_wait_ld();
#pragma unroll
                        for (int g = 0; g < 4; ++g) {
                            if (g >= nl) continue;
                            reg_after_wait(r[g]);
                            if (row_ok) store16(yrow, col0 + c0 + 16 * g, P.ldy, P.out_bf16, wide, r[g]);
                        }
                    }
                    epart();
                    fence_before();
                    mbar_arrive(&acc_empty[4 * buf + mt]);
                }
            }
        }
        if (lane == 0 && nst > 0) bulk_wait_all();   // every store has landed before the block exits
        if (!ok) atomicExch(err, 3);
    }
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TMEM_COLS));
    }
    // no block leaves while another may still multicast into it or arrive on its barriers
    cluster_sync_all();
}

// Pre-tile H_e (FP32, ne x ne per cell) into bf16 MMA blocks:
// [cell][s][mt][rg 16][kg 2][ri 8][ki 8].  Row R is the cell-local node
// (az*(p+1) + ay)*(p+1) + ax; column K = (z*(p+1) + y)*xpad + x follows the B
// rows, with zeros for the padding nodes x >= p+1 and outside ne x ne.
__global__ void k_tile_he16(int ncells, int np1, int xpad, int MT, int ksteps, const float *He32,
                            __nv_bfloat16 *He16) {
    const int ne = np1 * np1 * np1;
    const int krows = np1 * np1 * xpad;
    long long total = (long long)ncells * MT * ksteps * 2048;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int e = (int)(i % 2048);
        long long blk = i / 2048;
        int mt = (int)(blk % MT);
        int s = (int)((blk / MT) % ksteps);
        long long cell = blk / ((long long)ksteps * MT);
        int core = e / 64, within = e % 64;
        int rg = core / 2, kg = core % 2, ri = within / 8, ki = within % 8;
        int R = mt * 128 + rg * 8 + ri;
        int K = s * 16 + kg * 8 + ki;
        float v = 0.f;
        if (R < ne && K < krows) {
            int x = K % xpad, y = (K / xpad) % np1, z = K / (xpad * np1);
            if (x < np1) v = He32[(size_t)cell * ne * ne + (size_t)R * ne + (z * np1 + y) * np1 + x];
        }
        He16[i] = __float2bfloat16_rn(v);
    }
}

// The coupling's extra A stages of each cell, in the layout of the H_e tiles:
// stage j of cell c holds atom slots 2j, 2j+1 (columns 8 kg + ki: E_ki for
// ki < 4, P_c,ki-4 otherwise) at the rows of the interior nodes the cell owns
// (local indices in [0, p)^3); every other row is zero, so each FE row gets
// its coupling from exactly one cell.  Values from the node-major tables.
__global__ void k_tile_coupling(MeshDev m, int MT, const int *__restrict__ cx_off, const int *__restrict__ cx_atoms,
                                int natoms, const long long *__restrict__ node_ptr, const int *__restrict__ nm_atom,
                                const float *__restrict__ nmE, const float *__restrict__ nmP, int use_e, int use_p,
                                __nv_bfloat16 *__restrict__ Ax) {
    const int c = blockIdx.x;
    const int x0 = cx_off[c], nxs = cx_off[c + 1] - x0;
    const int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
    const long long total = (long long)nxs * MT * 2048;
    for (long long i = threadIdx.x; i < total; i += blockDim.x) {
        const int e = (int)(i % 2048);
        const long long blk = i / 2048;
        const int mt = (int)(blk % MT), j = (int)(blk / MT);
        const int core = e / 64, within = e % 64;
        const int rg = core / 2, kg = core % 2, ri = within / 8, ki = within % 8;
        const int R = mt * 128 + rg * 8 + ri;
        const int atom = cx_atoms[2 * (x0 + j) + kg];
        float v = 0.f;
        if (R < m.ne && atom < natoms) {
            const int ax = R % m.np1, ay = (R / m.np1) % m.np1, az = R / (m.np1 * m.np1);
            const int ix = cx * m.p + ax, iy = cy * m.p + ay, iz = cz * m.p + az;
            if (ax < m.p && ay < m.p && az < m.p && ix >= 1 && iy >= 1 && iz >= 1 && ix <= m.Gx - 2 &&
                iy <= m.Gy - 2 && iz <= m.Gz - 2) {
                const long long n = ((long long)iz * m.Gy + iy) * m.Gx + ix;
                for (long long q = node_ptr[n]; q < node_ptr[n + 1]; ++q)
                    if ((nm_atom[q] & kNmAtomMask) == atom) {
                        if (ki < 4) v = use_e ? nmE[4 * q + ki] : 0.f;
                        else v = use_p ? nmP[4 * q + ki - 4] : 0.f;
                        break;
                    }
            }
        }
        Ax[((size_t)(x0 + j) * MT + mt) * 2048 + e] = __float2bfloat16_rn(v);
    }
}

// The padding rows of each cell's last M-tile (rows ne .. MT*128): row
// ne + 4 s + f holds E_f of the cell's s-th support atom (the cell-atom list:
// the atoms whose support cells include the cell), as a row of the cell matrix
// over the operand's K ordering (node (z*(p+1) + y)*xpad + x), so the cell
// products also return the cell's share of E Y_c.  Each (node, atom) entry
// goes to exactly one cell: of the cells that contain the node and are
// support cells of the atom, the one with the largest index.  Zero elsewhere.
__global__ void k_tile_epad(MeshDev m, int MT, int xpad, int ksteps, const int *__restrict__ ca_ptr,
                            const int *__restrict__ ca_atoms, const long long *__restrict__ node_ptr,
                            const int *__restrict__ nm_atom, const float *__restrict__ nmE,
                            __nv_bfloat16 *__restrict__ He16) {
    const int c = blockIdx.x;
    const int q0 = ca_ptr[c], nslot = ca_ptr[c + 1] - q0;
    const int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
    const int mt = MT - 1, r0 = m.ne - mt * 128;         // first padding row within the tile
    const int nrow = 128 - r0;
    const long long total = (long long)ksteps * nrow * 16;
    for (long long i = threadIdx.x; i < total; i += blockDim.x) {
        const int kk = (int)(i % 16);
        const int rr = (int)((i / 16) % nrow);
        const int s = (int)(i / (16LL * nrow));
        const int Rt = r0 + rr;                           // row within the tile
        const int rg = Rt / 8, ri = Rt % 8, kg = kk / 8, ki = kk % 8;
        const int r = Rt + mt * 128 - m.ne, slot = r / 4, f = r % 4;
        float v = 0.f;
        if (slot < nslot) {
            const int atom = ca_atoms[q0 + slot];
            const int K = s * 16 + kk;
            const int x = K % xpad, y = (K / xpad) % m.np1, z = K / (xpad * m.np1);
            const int ix = cx * m.p + x, iy = cy * m.p + y, iz = cz * m.p + z;
            if (x < m.np1 && z < m.np1 && ix >= 1 && iy >= 1 && iz >= 1 && ix <= m.Gx - 2 && iy <= m.Gy - 2 &&
                iz <= m.Gz - 2) {
                // the largest-index support cell of `atom` containing the node
                int best = -1;
                for (int dz = 0; dz < 2; ++dz)
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            const int ex = ix / m.p - dx, ey = iy / m.p - dy, ez = iz / m.p - dz;
                            if (ex < 0 || ey < 0 || ez < 0 || ex >= m.nx || ey >= m.ny || ez >= m.nz) continue;
                            if (ix - ex * m.p > m.p || iy - ey * m.p > m.p || iz - ez * m.p > m.p) continue;
                            const int e = (ez * m.ny + ey) * m.nx + ex;
                            if (e <= best) continue;
                            for (int q = ca_ptr[e]; q < ca_ptr[e + 1]; ++q)
                                if (ca_atoms[q] == atom) { best = e; break; }
                        }
                if (best == c) {
                    const long long n = ((long long)iz * m.Gy + iy) * m.Gx + ix;
                    for (long long q = node_ptr[n]; q < node_ptr[n + 1]; ++q)
                        if ((nm_atom[q] & kNmAtomMask) == atom) {
                            v = nmE[4 * q + f];
                            break;
                        }
                }
            }
        }
        const size_t e = (((size_t)c * ksteps + s) * MT + mt) * 2048 + (size_t)(rg * 2 + kg) * 64 + ri * 8 + ki;
        He16[e] = __float2bfloat16_rn(v);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode(efe_ctx *ctx) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p) {
            ctx->err = "cuTensorMapEncodeTiled is not available";
            return nullptr;
        }
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

// Geometry of the tensor-core cell product for this mesh and N columns.
struct TcShape {
    int xpad, Kpad, ksteps, MT, Npad, nchunks, plane_rows, kpg, ngroups, a_stages, ks, slot_bytes, x_slot_bytes;
    size_t smem;
};

constexpr size_t TC_FIXED = (2 * MAX_A_STAGES + 2 * B_SLOTS + 18) * 8 + 64 + 1024;   // barriers, TMEM slot, alignment

// shared memory: A ring + two B slots + the coupling slot + epilogue staging +
// barriers (+ alignment slack) within 227 KB
static size_t tc_smem(const TcShape &s) {
    return (size_t)EPI_STAGE + (size_t)s.a_stages * s.ks * s.MT * 4096 + (size_t)B_SLOTS * s.slot_bytes +
           s.x_slot_bytes + TC_FIXED;
}

// x_slots: atom slots of the coupling per cell (0: no coupling)
static TcShape tc_shape(const efe_ctx *ctx, int N, int ldb, int x_slots = 0) {
    TcShape s{};
    const int ne = ctx->m.ne, np1 = ctx->m.np1;
    s.xpad = (np1 + 7) / 8 * 8;
    s.Kpad = (np1 * np1 * s.xpad + 15) / 16 * 16;
    s.ksteps = s.Kpad / 16;
    s.MT = (ne + 127) / 128;
    s.plane_rows = np1 * s.xpad;
    s.kpg = 2 * s.plane_rows / 16;
    s.ngroups = (np1 + 1) / 2;
    const int stage = s.MT * 4096;
    const size_t fixed = TC_FIXED + EPI_STAGE;
    int maxN = std::min(256, (TMEM_COLS / s.MT) / 16 * 16);
    // keep at least 4 A stages
    while (maxN > 16 && fixed + 4 * (size_t)stage + (size_t)B_SLOTS * (maxN / 8) * 2 * s.plane_rows * 16 +
                                (size_t)x_slots * (maxN / 8) * 128 >
                            (size_t)SMEM_LIMIT)
        maxN -= 16;
    int Nn = std::min(ldb, ((N + 15) / 16) * 16);
    s.nchunks = (Nn + maxN - 1) / maxN;
    s.Npad = ((Nn + s.nchunks - 1) / s.nchunks + 15) / 16 * 16;
    s.slot_bytes = (s.Npad / 8) * 2 * s.plane_rows * 16;
    s.x_slot_bytes = x_slots * (s.Npad / 8) * 128;
    const size_t used = fixed + (size_t)B_SLOTS * s.slot_bytes + s.x_slot_bytes;
    const size_t left = used < (size_t)SMEM_LIMIT ? (size_t)SMEM_LIMIT - used : 0;
    // A stages of ks k-steps: each stage costs one producer/MMA barrier round
    // trip, so as many k-steps per stage as still leave three stages in flight
    s.ks = 1;
    for (int ks = 4; ks >= 1; --ks)
        if (left / ((size_t)ks * stage) >= 3 || ks == 1) {
            s.ks = ks;
            break;
        }
    s.a_stages = (int)std::min<size_t>(MAX_A_STAGES, left / ((size_t)s.ks * stage));
    s.smem = tc_smem(s);
    return s;
}

// The static part of the coupling in the cell products: per cell the atoms
// with a coupling entry (E or P_c; all support entries) at an interior node
// the cell owns, sorted and padded to an even count with the zero block
// (index natoms), two per extra k-step.
static efe_status tc_coupling_structure(efe_ctx *ctx, int MT) {
    if (ctx->cx_built) return EFE_OK;
    const MeshDev &m = ctx->m;
    const long long nn = ctx->n_nodes, ns = ctx->sup_total;
    std::vector<long long> np(nn + 1);
    std::vector<int> na((size_t)std::max<long long>(ns, 1));
    EFE_CUDA(ctx, cudaMemcpy(np.data(), ctx->d_node_ptr, sizeof(long long) * (nn + 1), cudaMemcpyDeviceToHost));
    if (ns > 0) EFE_CUDA(ctx, cudaMemcpy(na.data(), ctx->d_nm_atom, sizeof(int) * ns, cudaMemcpyDeviceToHost));
    const int ncells = m.nx * m.ny * m.nz;
    std::vector<int> off(ncells + 1, 0), atoms, list;
    int maxs = 0;
    for (int c = 0; c < ncells; ++c) {
        const int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
        list.clear();
        for (int az = 0; az < m.p; ++az)
            for (int ay = 0; ay < m.p; ++ay)
                for (int ax = 0; ax < m.p; ++ax) {
                    const int ix = cx * m.p + ax, iy = cy * m.p + ay, iz = cz * m.p + az;
                    if (ix < 1 || iy < 1 || iz < 1 || ix > m.Gx - 2 || iy > m.Gy - 2 || iz > m.Gz - 2) continue;
                    const long long n = ((long long)iz * m.Gy + iy) * m.Gx + ix;
                    for (long long e = np[n]; e < np[n + 1]; ++e) list.push_back(na[e] & kNmAtomMask);
                }
        std::sort(list.begin(), list.end());
        list.erase(std::unique(list.begin(), list.end()), list.end());
        if (list.size() & 1) list.push_back(ctx->natoms);
        off[c + 1] = off[c] + (int)(list.size() / 2);
        atoms.insert(atoms.end(), list.begin(), list.end());
        maxs = std::max(maxs, (int)list.size());
    }
    if (atoms.empty()) atoms.assign(2, ctx->natoms);
    // E Y_c from the padding rows: a cell's rows carry the atoms whose support
    // cells include it (the cell-atom lists); per atom, its (cell, atom) pairs
    // in cell order, over which the partials are summed
    std::vector<int> cptr(ncells + 1), cat;
    EFE_CUDA(ctx, cudaMemcpy(cptr.data(), ctx->d_cell_atom_ptr, sizeof(int) * (ncells + 1), cudaMemcpyDeviceToHost));
    cat.resize(std::max(cptr[ncells], 1));
    if (cptr[ncells] > 0)
        EFE_CUDA(ctx, cudaMemcpy(cat.data(), ctx->d_cell_atoms, sizeof(int) * cptr[ncells], cudaMemcpyDeviceToHost));
    int maxca = 0;
    for (int c = 0; c < ncells; ++c) maxca = std::max(maxca, cptr[c + 1] - cptr[c]);
    std::vector<int> aoff(ctx->natoms + 2, 0), apairs;
    for (int q = 0; q < cptr[ncells]; ++q) aoff[cat[q] + 2]++;
    for (int I = 0; I < ctx->natoms; ++I) aoff[I + 2] += aoff[I + 1];
    apairs.resize(std::max(aoff[ctx->natoms + 1], 1));
    for (int q = 0; q < cptr[ncells]; ++q) apairs[aoff[cat[q] + 1]++] = q;
    aoff.pop_back();
    ctx->ca_pairs = cptr[ncells];
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_atom_pair_off, sizeof(int) * (ctx->natoms + 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_atom_pairs, sizeof(int) * apairs.size()));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_atom_pair_off, aoff.data(), sizeof(int) * (ctx->natoms + 1),
                             cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_atom_pairs, apairs.data(), sizeof(int) * apairs.size(), cudaMemcpyHostToDevice));
    // the padding rows hold 4 E rows per cell-atom pair when they suffice
    ctx->epad = ctx->enrich && 4 * maxca <= MT * 128 - m.ne;
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_cx_off, sizeof(int) * (ncells + 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_cx_atoms, sizeof(int) * atoms.size()));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_cx_off, off.data(), sizeof(int) * (ncells + 1), cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_cx_atoms, atoms.data(), sizeof(int) * atoms.size(), cudaMemcpyHostToDevice));
    ctx->cx_steps = off[ncells];
    EFE_TRY(efe_alloc(ctx, &ctx->d_Ax, sizeof(__nv_bfloat16) * (size_t)std::max(ctx->cx_steps, 1LL) * MT * 2048));
    ctx->cx_max_slots = maxs;
    ctx->cx_built = true;
    return EFE_OK;
}

// Per atom I, the atoms J whose 4x4 blocks of H^E_ee (I, J) or of P^E
// ((I, J) or (J, I)) hold a nonzero, read from the assembled FP64 blocks of
// the current potential (overlapping supports; I itself included).
static efe_status tc_block_pattern(efe_ctx *ctx) {
    const int na = ctx->natoms, ne = ctx->n_enr;
    std::vector<double> he, pe;
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->enrich) {
        he.resize((size_t)ne * ne);
        EFE_CUDA(ctx, cudaMemcpy(he.data(), ctx->d_HEee, sizeof(double) * he.size(), cudaMemcpyDeviceToHost));
        if (ctx->nonlocal && ctx->d_PE) {
            pe.resize((size_t)ctx->n_proj * ne);
            EFE_CUDA(ctx, cudaMemcpy(pe.data(), ctx->d_PE, sizeof(double) * pe.size(), cudaMemcpyDeviceToHost));
        }
    }
    std::vector<int> ptr(na + 1, 0), nb;
    for (int I = 0; I < na; ++I) {
        for (int J = 0; J < na; ++J) {
            bool nz = I == J;
            for (int a = 0; a < 4 && !nz; ++a)
                for (int b = 0; b < 4 && !nz; ++b) {
                    if (!he.empty() && he[(size_t)(4 * I + a) * ne + 4 * J + b] != 0.0) nz = true;
                    if (!pe.empty() && (pe[(size_t)(4 * I + a) * ne + 4 * J + b] != 0.0 ||
                                        pe[(size_t)(4 * J + a) * ne + 4 * I + b] != 0.0))
                        nz = true;
                }
            if (nz) nb.push_back(J);
        }
        ptr[I + 1] = (int)nb.size();
    }
    if (nb.empty()) nb.push_back(0);
    if (!ctx->d_enbr_ptr) EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_enbr_ptr, sizeof(int) * (na + 1)));
    if (ctx->d_enbr) cudaFree(ctx->d_enbr);
    ctx->d_enbr = nullptr;
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_enbr, sizeof(int) * nb.size()));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_enbr_ptr, ptr.data(), sizeof(int) * (na + 1), cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_enbr, nb.data(), sizeof(int) * nb.size(), cudaMemcpyHostToDevice));
    return EFE_OK;
}

efe_status efe_tc_prepare(efe_ctx *ctx) {
    const MeshDev &m = ctx->m;
    const int ne = m.ne;
    const int xpad = (m.np1 + 7) / 8 * 8;
    const int Kpad = (m.np1 * m.np1 * xpad + 15) / 16 * 16, MT = (ne + 127) / 128, ksteps = Kpad / 16;
    if (MT > 4) {
        ctx->err = "tensor-core cell product supports (p+1)^3 <= 512";
        return EFE_ERR_ARG;
    }
    const long long ncells = (long long)m.nx * m.ny * m.nz;
    const size_t bytes = (size_t)ncells * MT * ksteps * 2048 * sizeof(__nv_bfloat16);
    if (!ctx->d_He16) {
        EFE_TRY(efe_alloc(ctx, &ctx->d_He16, bytes));
        ctx->he16_bytes = bytes;
    }
    k_tile_he16<<<1024, 256, 0, ctx->stream>>>((int)ncells, m.np1, xpad, MT, ksteps, ctx->d_He32,
                                               reinterpret_cast<__nv_bfloat16 *>(ctx->d_He16));
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_tile_he16"));
    if ((ctx->enrich || ctx->nonlocal) && ctx->natoms > 0 && ctx->d_node_ptr && ctx->d_nm_atom) {
        EFE_TRY(tc_coupling_structure(ctx, MT));
        k_tile_coupling<<<(unsigned)ncells, 256, 0, ctx->stream>>>(
            m, MT, ctx->d_cx_off, ctx->d_cx_atoms, ctx->natoms, ctx->d_node_ptr, ctx->d_nm_atom, ctx->d_nm_E32,
            ctx->d_nm_P32, ctx->enrich ? 1 : 0, ctx->nonlocal ? 1 : 0, reinterpret_cast<__nv_bfloat16 *>(ctx->d_Ax));
        ctx->launches++;
        EFE_TRY(efe_check_launch(ctx, "k_tile_coupling"));
        EFE_TRY(tc_block_pattern(ctx));
        if (ctx->epad) {
            k_tile_epad<<<(unsigned)ncells, 256, 0, ctx->stream>>>(
                m, MT, xpad, ksteps, ctx->d_cell_atom_ptr, ctx->d_cell_atoms, ctx->d_node_ptr, ctx->d_nm_atom,
                ctx->d_nm_E32, reinterpret_cast<__nv_bfloat16 *>(ctx->d_He16));
            ctx->launches++;
            EFE_TRY(efe_check_launch(ctx, "k_tile_epad"));
        }
    }
    ctx->he16_valid = true;
    return EFE_OK;
}

// Columns of one row of the coupling table YW that the cell products may read
// for N columns of row stride ldb (all chunks): nchunks x Npad.
int efe_tc_columns(const efe_ctx *ctx, int N, int ldb) {
    const TcShape sh = tc_shape(ctx, N, ldb, ctx->cx_built ? ctx->cx_max_slots : 0);
    return sh.nchunks * sh.Npad;
}

// Ycells[cell][row][ldy] = H_e X'_e for all cells (FP32, or bf16 when out_bf16);
// X'_bf16: n_nodes x ldb.  With YW (the Y_e / W table, [natoms + 1][nCB][8][8]
// bf16, nCB = efe_tc_columns / 8, the last atom block zero) the owned FE rows
// of each cell also receive E^T Y_e + P_c^T W.
efe_status efe_tc_cells(efe_ctx *ctx, const void *Xp_bf16, int ldb, int N, void *Ycells, int ldy, int *d_err,
                        int out_bf16, const void *YW, int nCB, float *Epart) {
    const MeshDev &m = ctx->m;
    if (!ctx->he16_valid) EFE_TRY(efe_tc_prepare(ctx));
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode(ctx);
    if (!encode) return EFE_ERR_CUDA;
    alignas(64) CUtensorMap map;
    cuuint64_t gdim[4] = {(cuuint64_t)ldb, (cuuint64_t)m.Gx, (cuuint64_t)m.Gy, (cuuint64_t)m.Gz};
    cuuint64_t gstr[3] = {(cuuint64_t)ldb * 2, (cuuint64_t)ldb * 2 * m.Gx, (cuuint64_t)ldb * 2 * m.Gx * m.Gy};
    const bool cpl = YW && ctx->cx_built && ctx->cx_steps > 0;
    TcShape sh = tc_shape(ctx, N, ldb, cpl ? ctx->cx_max_slots : 0);
    cuuint32_t box[4] = {8, (cuuint32_t)sh.xpad, (cuuint32_t)m.np1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(Xp_bf16), gdim, gstr, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        ctx->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")";
        return EFE_ERR_CUDA;
    }
    const int ncells = m.nx * m.ny * m.nz;
    // bf16 output rows: Ycells as {ldy columns, n_e rows, cells}, stored by
    // 16 x 32 boxes (32-byte swizzle); rows past n_e fall outside the map
    // (TMA stores only where every box lies inside the rows' columns and the row
    // pitch is a whole number of 32-byte swizzle spans; otherwise direct stores)
    alignas(64) CUtensorMap ymap;
    std::memset(&ymap, 0, sizeof(ymap));
    const bool tma_out = out_bf16 && ldy % 16 == 0 && sh.nchunks * sh.Npad <= ldy &&
                         (reinterpret_cast<uintptr_t>(Ycells) & 15) == 0;
    if (tma_out) {
        cuuint64_t ydim[3] = {(cuuint64_t)ldy, (cuuint64_t)m.ne, (cuuint64_t)ncells};
        cuuint64_t ystr[2] = {(cuuint64_t)ldy * 2, (cuuint64_t)ldy * 2 * m.ne};
        cuuint32_t ybox[3] = {16, 32, 1};
        cuuint32_t yes[3] = {1, 1, 1};
        cr = encode(&ymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, Ycells, ydim, ystr, ybox, yes,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            ctx->err = "cuTensorMapEncodeTiled failed for the output rows (" + std::to_string((int)cr) + ")";
            return EFE_ERR_CUDA;
        }
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    TcParams P{};
    P.ncells = ncells;
    P.nx = m.nx;
    P.ny = m.ny;
    P.p = m.p;
    P.np1 = m.np1;
    P.ne = m.ne;
    P.xpad = sh.xpad;
    P.Kpad = sh.Kpad;
    P.ksteps = sh.ksteps;
    P.MT = sh.MT;
    P.Npad = sh.Npad;
    P.ncb = sh.Npad / 8;
    P.ldy = ldy;
    P.plane_rows = sh.plane_rows;
    P.kpg = sh.kpg;
    P.ngroups = sh.ngroups;
    P.a_stages = sh.a_stages;
    P.ks = sh.ks;
    P.slot_bytes = sh.slot_bytes;
    P.out_bf16 = out_bf16;
    P.cx_off = cpl ? ctx->d_cx_off : nullptr;
    P.cx_atoms = cpl ? ctx->d_cx_atoms : nullptr;
    P.Ax = reinterpret_cast<const __nv_bfloat16 *>(ctx->d_Ax);
    P.YW = reinterpret_cast<const __nv_bfloat16 *>(YW);
    P.nCB = nCB;
    P.x_slot_bytes = sh.x_slot_bytes;
    P.Epart = (cpl && ctx->epad) ? Epart : nullptr;
    P.ca_ptr = ctx->d_cell_atom_ptr;
    P.tma_out = tma_out ? 1 : 0;
    if (cpl && sh.nchunks * P.ncb > nCB) {
        ctx->err = "tensor-core cell product: coupling table narrower than the column chunks";
        return EFE_ERR_ARG;
    }
    P.ncl = sh.nchunks;
    P.nbuf = 2 * sh.MT * sh.Npad <= TMEM_COLS ? 2 : 1;
    if (sh.a_stages < 2 || sh.smem > (size_t)SMEM_LIMIT || sh.MT * sh.Npad > TMEM_COLS || sh.nchunks > 8) {
        ctx->err = "tensor-core cell product: shared- or tensor-memory plan does not fit";
        return EFE_ERR_ARG;
    }
    // more than half of an SM's shared memory: one block per SM, so that no two
    // blocks (of one cluster, or not) compete for the SM's 512 TMEM columns
    const size_t shm = std::max(sh.smem, (size_t)120 * 1024);
    EFE_CUDA(ctx, cudaFuncSetAttribute(k_cell_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    // one block per SM; a cluster of nchunks blocks (x, 0..nchunks-1) walks the
    // same cells, one column chunk each; as many clusters as fit at once
    const int sms = nsm > 0 ? nsm : 148;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = (unsigned)sh.nchunks;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = shm;
    cfg.stream = ctx->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int gx = std::max(1, sms / sh.nchunks);
    cfg.gridDim = dim3((unsigned)gx, (unsigned)sh.nchunks);
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_cell_mma, &cfg) == cudaSuccess && nclusters > 0)
        gx = std::min(gx, nclusters);
    gx = std::max(1, std::min(gx, ncells));
    cfg.gridDim = dim3((unsigned)gx, (unsigned)sh.nchunks);
    EFE_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_cell_mma, map, ymap, reinterpret_cast<const __nv_bfloat16 *>(ctx->d_He16),
                                     Ycells, P, d_err));
    ctx->launches++;
    ctx->cell_launches++;
    EFE_TRY(efe_check_launch(ctx, "k_cell_mma"));
    return EFE_OK;
}
