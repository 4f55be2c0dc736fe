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
// freed shared memory deepens the A ring; the epilogue of a cell overlaps the
// loads of the next.
// Per-cell results go to Ycells[cell][row][ldy] (FP32); a gather kernel sums
// the up-to-8 contributions of each node, so no colouring or atomics are
// needed and every cell of the mesh runs in one persistent launch.
#include "efe_internal.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>

namespace {

constexpr int TC_THREADS = 256;      // w0 TMA producer, w1 MMA issuer, w2 TMEM owner, w4-7 epilogue
constexpr int MAX_A_STAGES = 24;     // A ring depth limit (one stage = one k-step of all M-tiles)
constexpr int B_SLOTS = 2;           // plane-pair ring
constexpr int SMEM_LIMIT = 232448;   // dynamic shared memory per block (227 KB)
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz before a wait gives up

struct TcParams {
    int ncells, nx, ny, p, np1, ne, xpad, Kpad, ksteps, MT, Npad, ncb, col0, ldy;
    int plane_rows;                     // (p+1) xpad rows per z-plane
    int kpg;                            // k-steps per plane pair: 2 plane_rows / 16
    int ngroups;                        // plane pairs per cell: ceil((p+1) / 2)
    int a_stages;                       // A ring depth
    int slot_bytes;                     // one B slot: ncb x 2 plane_rows x 16 B
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

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_cell_mma(const __grid_constant__ CUtensorMap xmap, const __nv_bfloat16 *__restrict__ He16, float *Ycells,
               TcParams P, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // every TMA destination below is a multiple of 128 B from this base
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    const int stage_bytes = P.MT * 4096;
    unsigned char *sA = smem;
    unsigned char *sB = smem + (size_t)P.a_stages * stage_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)B_SLOTS * P.slot_bytes);
    uint64_t *full_a = bars, *empty_a = bars + MAX_A_STAGES;
    uint64_t *full_b = bars + 2 * MAX_A_STAGES, *empty_b = full_b + B_SLOTS;
    uint64_t *acc_full = empty_b + B_SLOTS, *acc_empty = acc_full + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair_stride = 2 * P.plane_rows * 16;   // bytes between column blocks in a slot

    if (threadIdx.x == 0) {
        for (int i = 0; i < P.a_stages; ++i) { mbar_init(&full_a[i], 1); mbar_init(&empty_a[i], 1); }
        for (int i = 0; i < B_SLOTS; ++i) { mbar_init(&full_b[i], 1); mbar_init(&empty_b[i], 1); }
        for (int t = 0; t < 4; ++t) { mbar_init(&acc_full[t], 1); mbar_init(&acc_empty[t], 128); }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // zero both B slots once: rows a lone last plane leaves unwritten meet zero
    // columns of H_e, and must hold finite values
    for (int i = threadIdx.x; i < B_SLOTS * P.slot_bytes / 4; i += blockDim.x)
        reinterpret_cast<uint32_t *>(sB)[i] = 0u;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
        fence_before();
    }
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ---------------- producer ----------------
        int sa = 0, sb = 0;
        uint32_t pha = 0, phb = 0;
        bool ok = true;
        uint32_t aused = 0, apar = 0;      // per A slot: issued at least once, parity of its last phase
        uint32_t bused = 0, bpar = 0;      // the same per B slot
        for (int cell = blockIdx.x; cell < P.ncells && ok; cell += gridDim.x) {
            const int cx = cell % P.nx, cy = (cell / P.nx) % P.ny, cz = cell / (P.nx * P.ny);
            const __nv_bfloat16 *Ac = He16 + (size_t)cell * P.ksteps * P.MT * 2048;
            int s = 0;
            for (int g = 0; g < P.ngroups && ok; ++g) {
                // plane pair g -> B slot sb
                if (!mbar_wait(&empty_b[sb], phb ^ 1)) { ok = false; break; }
                const int np = min(2, P.np1 - 2 * g);
                mbar_expect_tx(&full_b[sb], (uint32_t)(np * P.plane_rows * 16 * P.ncb));
                unsigned char *slot = sB + (size_t)sb * P.slot_bytes;
                for (int zz = 0; zz < np; ++zz)
                    for (int cb = 0; cb < P.ncb; ++cb)
                        tma_load_4d(slot + (size_t)cb * pair_stride + (size_t)zz * P.plane_rows * 16, &xmap,
                                    P.col0 + 8 * cb, cx * P.p, cy * P.p, cz * P.p + 2 * g + zz,
                                    &full_b[sb]);   // {cols, x, y, z}
                bused |= 1u << sb;
                bpar = (bpar & ~(1u << sb)) | (phb << sb);
                if (++sb == B_SLOTS) { sb = 0; phb ^= 1; }
                // the A stages of this pair's k-steps
                const int s_end = min(P.ksteps, (g + 1) * P.kpg);
                for (; s < s_end; ++s) {
                    if (!mbar_wait(&empty_a[sa], pha ^ 1)) { ok = false; break; }
                    mbar_expect_tx(&full_a[sa], (uint32_t)stage_bytes);
                    bulk_load(sA + (size_t)sa * stage_bytes, Ac + (size_t)s * P.MT * 2048, (uint32_t)stage_bytes,
                              &full_a[sa]);
                    aused |= 1u << sa;
                    apar = (apar & ~(1u << sa)) | (pha << sa);
                    if (++sa == P.a_stages) { sa = 0; pha ^= 1; }
                }
            }
        }
        if (!ok) atomicExch(err, 1);
        // drain: every copy this thread issued has landed before the block exits
        for (int i = 0; i < B_SLOTS; ++i)
            if (bused & (1u << i)) mbar_wait(&full_b[i], (bpar >> i) & 1u);
        for (int i = 0; i < P.a_stages; ++i)
            if (aused & (1u << i)) mbar_wait(&full_a[i], (apar >> i) & 1u);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (0u << 15) | (1u << 16) |
                               ((uint32_t)(P.Npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        int sa = 0, sb = 0;
        uint32_t pha = 0, phb = 0;
        int it = 0;
        bool ok = true;
        const uint32_t sB_addr = smem_u32(sB), sA_addr = smem_u32(sA);
        for (int cell = blockIdx.x; cell < P.ncells && ok; cell += gridDim.x, ++it) {
            // every M-tile accumulates over the whole cell: all of them must be drained
            for (int mt = 0; mt < P.MT && ok; ++mt)
                if (!mbar_wait(&acc_empty[mt], (it & 1) ^ 1)) ok = false;
            if (!ok) break;
            fence_after();
            for (int s = 0; s < P.ksteps; ++s) {
                const int g = s / P.kpg, j = s - g * P.kpg;
                if (j == 0) {
                    if (!mbar_wait(&full_b[sb], phb)) { ok = false; break; }
                    fence_after();
                }
                if (!mbar_wait(&full_a[sa], pha)) { ok = false; break; }
                fence_after();
                const uint64_t bd = smem_desc(sB_addr + sb * P.slot_bytes + j * 256, 128, (uint32_t)pair_stride);
                for (int mt = 0; mt < P.MT; ++mt) {
                    const uint64_t ad = smem_desc(sA_addr + sa * stage_bytes + mt * 4096, 128, 256);
                    mma_bf16(tmem + (uint32_t)(mt * P.Npad), ad, bd, idesc, s > 0 ? 1u : 0u);
                }
                mma_commit(&empty_a[sa]);
                if (++sa == P.a_stages) { sa = 0; pha ^= 1; }
                if (j == P.kpg - 1 || s == P.ksteps - 1) {
                    mma_commit(&empty_b[sb]);
                    if (++sb == B_SLOTS) { sb = 0; phb ^= 1; }
                }
            }
            if (!ok) break;
            for (int mt = 0; mt < P.MT; ++mt) mma_commit(&acc_full[mt]);
        }
        if (!ok) atomicExch(err, 2);
    } else if (warp >= 4) {
        // ---------------- epilogue ----------------
        const int q = warp & 3;
        int it = 0;
        bool ok = true;
        for (int cell = blockIdx.x; cell < P.ncells && ok; cell += gridDim.x, ++it) {
            for (int mt = 0; mt < P.MT; ++mt) {
                // warp-uniform decision: the TMEM loads below are .sync.aligned
                const bool got = mbar_wait(&acc_full[mt], it & 1);
                if (!__all_sync(0xffffffffu, got)) { ok = false; break; }
                fence_after();
                const int row = mt * 128 + q * 32 + lane;
                float *dst = Ycells + ((size_t)cell * P.ne + row) * P.ldy + P.col0;
                const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(mt * P.Npad);
                // up to 64 columns per TMEM round trip: four loads, one wait
                for (int c = 0; c < P.Npad; c += 64) {
                    const int ng = min(4, (P.Npad - c) / 16);        // warp-uniform
                    uint32_t r[4][16];
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        if (g < ng) tmem_ld16_nw(tbase + (uint32_t)(c + 16 * g), r[g]);
                    tmem_wait_ld();
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                        if (g >= ng) continue;
                        reg_after_wait(r[g]);
                        if (row < P.ne) {
                            const int cc = c + 16 * g;
#pragma unroll
                            for (int i = 0; i < 16; i += 4)
                                if (P.col0 + cc + i + 3 < P.ldy)
                                    *reinterpret_cast<float4 *>(dst + cc + i) =
                                        make_float4(__uint_as_float(r[g][i]), __uint_as_float(r[g][i + 1]),
                                                    __uint_as_float(r[g][i + 2]), __uint_as_float(r[g][i + 3]));
                        }
                    }
                }
                fence_before();
                mbar_arrive(&acc_empty[mt]);
            }
        }
        if (!ok) atomicExch(err, 3);
    }
    __syncthreads();
    if (warp == 2) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
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
    int xpad, Kpad, ksteps, MT, Npad, nchunks, plane_rows, kpg, ngroups, a_stages, slot_bytes;
    size_t smem;
};

// shared memory: A ring + two B slots + barriers (+ alignment slack) within 227 KB
static size_t tc_smem(const TcShape &s) {
    return (size_t)s.a_stages * s.MT * 4096 + (size_t)B_SLOTS * s.slot_bytes +
           (2 * MAX_A_STAGES + 2 * B_SLOTS + 8) * 8 + 64 + 1024;
}

static TcShape tc_shape(const efe_ctx *ctx, int N, int ldb) {
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
    const size_t fixed = (2 * MAX_A_STAGES + 2 * B_SLOTS + 8) * 8 + 64 + 1024;
    int maxN = std::min(256, (512 / s.MT) / 16 * 16);
    // keep at least 4 A stages
    while (maxN > 16 && fixed + 4 * (size_t)stage + (size_t)B_SLOTS * (maxN / 8) * 2 * s.plane_rows * 16 >
                            (size_t)SMEM_LIMIT)
        maxN -= 16;
    int Nn = std::min(ldb, ((N + 15) / 16) * 16);
    s.nchunks = (Nn + maxN - 1) / maxN;
    s.Npad = ((Nn + s.nchunks - 1) / s.nchunks + 15) / 16 * 16;
    s.slot_bytes = (s.Npad / 8) * 2 * s.plane_rows * 16;
    const size_t left = (size_t)SMEM_LIMIT - fixed - (size_t)B_SLOTS * s.slot_bytes;
    s.a_stages = (int)std::min<size_t>(MAX_A_STAGES, left / stage);
    s.smem = tc_smem(s);
    return s;
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
    ctx->he16_valid = true;
    return EFE_OK;
}

// Ycells[cell][row][ldy] = H_e X'_e for all cells; X'_bf16: n_nodes x ldb.
efe_status efe_tc_cells(efe_ctx *ctx, const void *Xp_bf16, int ldb, int N, float *Ycells, int ldy, int *d_err) {
    const MeshDev &m = ctx->m;
    if (!ctx->he16_valid) EFE_TRY(efe_tc_prepare(ctx));
    PFN_cuTensorMapEncodeTiled_v12000 encode = get_encode(ctx);
    if (!encode) return EFE_ERR_CUDA;
    alignas(64) CUtensorMap map;
    cuuint64_t gdim[4] = {(cuuint64_t)ldb, (cuuint64_t)m.Gx, (cuuint64_t)m.Gy, (cuuint64_t)m.Gz};
    cuuint64_t gstr[3] = {(cuuint64_t)ldb * 2, (cuuint64_t)ldb * 2 * m.Gx, (cuuint64_t)ldb * 2 * m.Gx * m.Gy};
    TcShape sh = tc_shape(ctx, N, ldb);
    cuuint32_t box[4] = {8, (cuuint32_t)sh.xpad, (cuuint32_t)m.np1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(Xp_bf16), gdim, gstr, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        ctx->err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)cr) + ")";
        return EFE_ERR_CUDA;
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int ncells = m.nx * m.ny * m.nz;
    for (int ch = 0; ch < sh.nchunks; ++ch) {
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
        P.col0 = ch * sh.Npad;
        P.ldy = ldy;
        P.plane_rows = sh.plane_rows;
        P.kpg = sh.kpg;
        P.ngroups = sh.ngroups;
        P.a_stages = sh.a_stages;
        P.slot_bytes = sh.slot_bytes;
        if (sh.a_stages < 4 || sh.smem > (size_t)SMEM_LIMIT) {
            ctx->err = "tensor-core cell product: shared-memory plan does not fit";
            return EFE_ERR_ARG;
        }
        const size_t shm = sh.smem;
        EFE_CUDA(ctx, cudaFuncSetAttribute(k_cell_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        const int grid = std::min(nsm > 0 ? nsm : 148, ncells);
        k_cell_mma<<<grid, TC_THREADS, shm, ctx->stream>>>(map, reinterpret_cast<const __nv_bfloat16 *>(ctx->d_He16),
                                                          Ycells, P, d_err);
        ctx->launches++;
        ctx->cell_launches++;
        EFE_TRY(efe_check_launch(ctx, "k_cell_mma"));
    }
    return EFE_OK;
}
