// H^E, M^E, (M~^E)^-1 products, the residual Chebyshev filter, Rayleigh-Ritz,
// Lanczos bounds and the C ABI entry points (paper Sec. II.B, III.A, III.B).
#include "efe_internal.cuh"
#include "efe_convert.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>

namespace {

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ inline bool node_interior(const MeshDev &m, int ix, int iy, int iz) {
    return ix > 0 && iy > 0 && iz > 0 && ix < m.Gx - 1 && iy < m.Gy - 1 && iz < m.Gz - 1;
}

// ---------------------------------------------------------------------------
// Cell products of one colour: Y[nodes(c)] += H_c X[nodes(c)].  Cells of one
// colour (parity of cx, cy, cz) share no node, so the read-modify-write of Y
// needs no atomics.  Block = one cell x TN columns; the cell's X block is
// gathered into shared memory by index arithmetic on the node grid.
// ---------------------------------------------------------------------------
template <typename T, int TN>
__global__ void __launch_bounds__(256) k_cell_apply(MeshDev m, int colour, const T *He, long long he_stride,
                                                    const T *X, T *Y, int N, int ld) {
    extern __shared__ unsigned char smraw[];
    T *sX = reinterpret_cast<T *>(smraw);
    const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
    const int hx = (m.nx - ox + 1) / 2, hy = (m.ny - oy + 1) / 2;
    const int b = blockIdx.x;
    const int cx = 2 * (b % hx) + ox, cy = 2 * ((b / hx) % hy) + oy, cz = 2 * (b / (hx * hy)) + oz;
    const int c = (cz * m.ny + cy) * m.nx + cx;
    const int col0 = blockIdx.y * TN;
    const int np1 = m.np1, ne = m.ne;
    for (int i = threadIdx.x; i < ne * TN; i += blockDim.x) {
        int l = i / TN, j = i % TN;
        int lx = l % np1, ly = (l / np1) % np1, lz = l / (np1 * np1);
        long long n = ((long long)(cz * m.p + lz) * m.Gy + (cy * m.p + ly)) * m.Gx + (cx * m.p + lx);
        sX[i] = (col0 + j < N) ? X[n * ld + col0 + j] : T(0);
    }
    __syncthreads();
    const T *H = He + (long long)c * he_stride;
    for (int i = threadIdx.x; i < ne * TN; i += blockDim.x) {
        int l = i / TN, j = i % TN;
        if (col0 + j >= N) continue;
        const T *Hr = H + (long long)l * ne;
        T acc = T(0);
        for (int k = 0; k < ne; ++k) acc += Hr[k] * sX[k * TN + j];
        int lx = l % np1, ly = (l / np1) % np1, lz = l / (np1 * np1);
        int ix = cx * m.p + lx, iy = cy * m.p + ly, iz = cz * m.p + lz;
        if (!node_interior(m, ix, iy, iz)) continue;
        long long n = ((long long)iz * m.Gy + iy) * m.Gx + ix;
        Y[n * ld + col0 + j] += acc;
    }
}

// events bracketing one sweep of cell products (reused across calls)
std::pair<cudaEvent_t, cudaEvent_t> *cell_event_pair(efe_ctx *ctx) {
    if (ctx->cell_events_used == ctx->cell_events.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return nullptr; }
        ctx->cell_events.push_back({a, b});
    }
    return &ctx->cell_events[ctx->cell_events_used++];
}

std::pair<cudaEvent_t, cudaEvent_t> *rec_event_pair(efe_ctx *ctx) {
    if (ctx->rec_events_used == ctx->rec_events.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return nullptr; }
        ctx->rec_events.push_back({a, b});
    }
    return &ctx->rec_events[ctx->rec_events_used++];
}

double rec_events_ms(efe_ctx *ctx) {
    double t = 0.0;
    for (size_t i = 0; i < ctx->rec_events_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->rec_events[i].first, ctx->rec_events[i].second) == cudaSuccess) t += ms;
    }
    ctx->rec_events_used = 0;
    return t;
}

// sum of the recorded sweeps (the stream must have been synchronised)
double cell_events_ms(efe_ctx *ctx) {
    double t = 0.0;
    for (size_t i = 0; i < ctx->cell_events_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->cell_events[i].first, ctx->cell_events[i].second) == cudaSuccess) t += ms;
    }
    ctx->cell_events_used = 0;
    return t;
}

template <typename T>
efe_status launch_cells(efe_ctx *ctx, const T *He, long long he_stride, const T *X, T *Y, int N, int ld,
                        bool timed = true) {
    const MeshDev &m = ctx->m;
    auto *ev = timed ? cell_event_pair(ctx) : nullptr;
    if (ev) cudaEventRecord(ev->first, ctx->stream);
    for (int colour = 0; colour < 8; ++colour) {
        const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
        const int hx = (m.nx - ox + 1) / 2, hy = (m.ny - oy + 1) / 2, hz = (m.nz - oz + 1) / 2;
        const int ncol = hx * hy * hz;
        if (!ncol) continue;
        if (N <= 8) {
            dim3 g(ncol, nblk(N, 8));
            size_t shm = sizeof(T) * m.ne * 8;
            cudaFuncSetAttribute(k_cell_apply<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            k_cell_apply<T, 8><<<g, 256, shm, ctx->stream>>>(m, colour, He, he_stride, X, Y, N, ld);
        } else if (N <= 16) {
            dim3 g(ncol, nblk(N, 16));
            size_t shm = sizeof(T) * m.ne * 16;
            cudaFuncSetAttribute(k_cell_apply<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            k_cell_apply<T, 16><<<g, 256, shm, ctx->stream>>>(m, colour, He, he_stride, X, Y, N, ld);
        } else {
            dim3 g(ncol, nblk(N, 32));
            size_t shm = sizeof(T) * m.ne * 32;
            cudaFuncSetAttribute(k_cell_apply<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            k_cell_apply<T, 32><<<g, 256, shm, ctx->stream>>>(m, colour, He, he_stride, X, Y, N, ld);
        }
        ctx->launches++;
        ctx->cell_launches++;
        EFE_TRY(efe_check_launch(ctx, "k_cell_apply"));
    }
    if (ev) cudaEventRecord(ev->second, ctx->stream);
    return EFE_OK;
}

// X'_c = X_c - C^T X_e (first half of T), boundary rows forced to zero.
template <typename T>
__global__ void k_xprime(MeshDev m, long long n_nodes, const T *X, T *Xp, int N, int ld,
                         const long long *node_ptr, const int *node_ent, const int *ent_atom,
                         const double *C, int use_c) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n_nodes * N) return;
    long long n = idx / N;
    int j = (int)(idx % N);
    int ix = (int)(n % m.Gx), iy = (int)((n / m.Gx) % m.Gy), iz = (int)(n / ((long long)m.Gx * m.Gy));
    if (!node_interior(m, ix, iy, iz)) { Xp[n * ld + j] = T(0); return; }
    T v = X[n * ld + j];
    if (use_c) {
        const T *Xe = X + n_nodes * ld;
        double acc = 0.0;
        for (long long e = node_ptr[n]; e < node_ptr[n + 1]; ++e) {
            int g = node_ent[e];
            int I = ent_atom[g];
            const double *c = C + 4 * (long long)g;
            acc += c[0] * (double)Xe[(4 * I + 0) * (long long)ld + j] + c[1] * (double)Xe[(4 * I + 1) * (long long)ld + j] +
                   c[2] * (double)Xe[(4 * I + 2) * (long long)ld + j] + c[3] * (double)Xe[(4 * I + 3) * (long long)ld + j];
        }
        v = (T)((double)v - acc);
    }
    Xp[n * ld + j] = v;
}

__device__ inline double to_d(double x) { return x; }
__device__ inline double to_d(float x) { return (double)x; }
__device__ inline double to_d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }

// Partial support reductions: for atom I (blockIdx.y) and chunk blockIdx.x,
//   part[(I*nch + chunk)][r][j] = sum_{g in chunk} coef_r[g] * S[node(g)][j]
// with up to 8 coefficient rows (two 4-wide tables A and B).
template <typename T>
__global__ void k_support_reduce(const long long *sup_off, const int *sup_node, const double *coefA,
                                 const double *coefB, const T *S, int N, int ld, int chunk, int nch,
                                 double *part) {
    const int I = blockIdx.y;
    const long long beg = sup_off[I] + (long long)blockIdx.x * chunk;
    const long long end = min(sup_off[I + 1], beg + chunk);
    const int nr = coefB ? 8 : 4;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (long long g = beg; g < end; ++g) {
            double s = to_d(S[(long long)sup_node[g] * ld + j]);
            const double *a = coefA + 4 * g;
            acc[0] += a[0] * s; acc[1] += a[1] * s; acc[2] += a[2] * s; acc[3] += a[3] * s;
            if (coefB) {
                const double *b2 = coefB + 4 * g;
                acc[4] += b2[0] * s; acc[5] += b2[1] * s; acc[6] += b2[2] * s; acc[7] += b2[3] * s;
            }
        }
        double *o = part + ((long long)(I * nch + blockIdx.x) * 8) * N;
        for (int r = 0; r < nr; ++r) o[(long long)r * N + j] = acc[r];
    }
}

// Sum the chunk partials: outA[4I+f][j] (rows 0-3) and outB[4I+f][j] (rows 4-7).
// nr = 8, or 4 when only rows 0-3 were formed.
__global__ void k_support_sum(int natoms, int nch, int N, const double *part, double *outA, double *outB,
                              int nr = 8) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)natoms * nr * N) return;
    int j = (int)(idx % N);
    int r = (int)((idx / N) % nr);
    int I = (int)(idx / ((long long)nr * N));
    double s = 0.0;
    for (int ch = 0; ch < nch; ++ch) s += part[((long long)(I * nch + ch) * 8 + r) * N + j];
    if (r < 4) { if (outA) outA[(long long)(4 * I + r) * N + j] = s; }
    else if (outB) outB[(long long)(4 * I + r - 4) * N + j] = s;
}

// E Y_c per atom from the padding-row partials of the cell products:
// Rh[4I + f][j] = sum over the atom's (cell, atom) pairs q of Epart[4q + f][j].
// Block = (atom, f, 32 columns); 8 lanes per column take every 8th pair
// (FP32 sums), then a fixed-order FP64 sum over the lanes (deterministic).
__global__ void __launch_bounds__(256) k_epart_sum(int N, int ld, const int *pair_off, const int *pairs,
                                                   const float *Epart, double *Rh) {
    __shared__ double red[8][32];
    const int I = blockIdx.z, f = blockIdx.y, j = blockIdx.x * 32 + (threadIdx.x & 31), pl = threadIdx.x >> 5;
    // each lane's share in FP32 (the partials are FP32; FP64 adds and widenings
    // per element would run on the narrow FP64 pipe), the 8 lanes in FP64
    float acc = 0.f;
    if (j < N)
        for (int q = pair_off[I] + pl; q < pair_off[I + 1]; q += 8)
            acc += Epart[((size_t)pairs[q] * 4 + f) * ld + j];
    red[pl][threadIdx.x & 31] = (double)acc;
    __syncthreads();
    if (pl == 0 && j < N) {
        const int t = threadIdx.x & 31;
        Rh[(size_t)(4 * I + f) * N + j] = ((red[0][t] + red[1][t]) + (red[2][t] + red[3][t])) +
                                          ((red[4][t] + red[5][t]) + (red[6][t] + red[7][t]));
    }
}

// W = D (Wc + Pa X_e)  (nonlocal strengths applied)
template <typename T>
__global__ void k_proj_w(int n_proj, int n_enr, const double *Wc, const double *Pa, const T *Xe, int ld,
                         const double *D, int N, double *W) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n_proj * N) return;
    int p = (int)(idx / N), j = (int)(idx % N);
    double s = Wc[idx];
    if (Pa)
        for (int k = 0; k < n_enr; ++k) s += Pa[(long long)p * n_enr + k] * (double)Xe[(long long)k * ld + j];
    W[idx] = D[p] * s;
}

// Y_e,raw = R_hac + H_aa X_e + Pa^T W
template <typename T>
__global__ void k_enr_raw(int n_enr, int n_proj, const double *Rhac, const double *Haa, const double *Pa,
                          const double *W, const T *Xe, int ld, int N, double *Ye) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n_enr * N) return;
    int k = (int)(idx / N), j = (int)(idx % N);
    double s = Rhac[idx];
    for (int k2 = 0; k2 < n_enr; ++k2) s += Haa[(long long)k * n_enr + k2] * (double)Xe[(long long)k2 * ld + j];
    if (Pa)
        for (int p = 0; p < n_proj; ++p) s += Pa[(long long)p * n_enr + k] * W[(long long)p * N + j];
    Ye[idx] = s;
}

// The same two products restricted to the nonzero atom blocks: nb_ptr/nb list,
// per atom I, the atoms J whose blocks (I, J) of H^E_ee or of P^E (either
// orientation) are not all zero (supports that overlap); exact zeros skipped.
template <typename T>
__global__ void k_proj_w_sp(int n_proj, int n_enr, const double *Wc, const double *Pa, const T *Xe, int ld,
                            const double *D, int N, const int *nb_ptr, const int *nb, double *W) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n_proj * N) return;
    const int p = (int)(idx / N), j = (int)(idx % N), I = p / 4;
    double s = Wc[idx];
    if (Pa)
        for (int q = nb_ptr[I]; q < nb_ptr[I + 1]; ++q) {
            const int k0 = 4 * nb[q];
#pragma unroll
            for (int g = 0; g < 4; ++g) s += Pa[(long long)p * n_enr + k0 + g] * (double)Xe[(long long)(k0 + g) * ld + j];
        }
    W[idx] = D[p] * s;
}

// The enriched rows of the bf16 filter over the nonzero atom blocks,
// Ye = Rhac + H^E_ee Xe + P^E^T W, in FP32 arithmetic (those rows are FP32):
// FP32 copies of H^E_ee and P^E, W as FP32 rows of stride ldw; Rhac read and
// Ye written in FP64 (one conversion each).
__global__ void k_enr_raw_f(int n_enr, const double *Rhac, const float *Haa, const float *Pa, const float *W, int ldw,
                            const float *Xe, int ld, int N, const int *nb_ptr, const int *nb, double *Ye) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n_enr * N) return;
    const int k = (int)(idx / N), j = (int)(idx % N), I = k / 4;
    float s = (float)Rhac[idx];
    for (int q = nb_ptr[I]; q < nb_ptr[I + 1]; ++q) {
        const int k0 = 4 * nb[q];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            s = fmaf(Haa[(long long)k * n_enr + k0 + g], Xe[(long long)(k0 + g) * ld + j], s);
            if (Pa) s = fmaf(Pa[(long long)(k0 + g) * n_enr + k], W[(long long)(k0 + g) * ldw + j], s);
        }
    }
    Ye[idx] = (double)s;
}
__global__ void k_d2f(long long n, const double *x, float *y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

// Y_c[n] += sum_entries (Hca X_e + Pc W)
template <typename T>
__global__ void k_node_coupling(long long n_nodes, const long long *node_ptr, const int *node_ent,
                                const int *ent_atom, const double *Hca, const double *Pc, const T *Xe,
                                int ld, const double *W, int N, T *Y, int use_h, int use_p) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n_nodes * N) return;
    long long n = idx / N;
    int j = (int)(idx % N);
    long long e0 = node_ptr[n], e1 = node_ptr[n + 1];
    if (e0 == e1) return;
    double acc = 0.0;
    for (long long e = e0; e < e1; ++e) {
        int g = node_ent[e];
        int I = ent_atom[g];
        if (use_h) {
            const double *h = Hca + 4 * (long long)g;
            for (int f = 0; f < 4; ++f) acc += h[f] * (double)Xe[(long long)(4 * I + f) * ld + j];
        }
        if (use_p) {
            const double *pc = Pc + 4 * (long long)g;
            for (int f = 0; f < 4; ++f) acc += pc[f] * W[(long long)(4 * I + f) * N + j];
        }
    }
    Y[n * ld + j] = (T)((double)Y[n * ld + j] + acc);
}

// Y_e = Y_e,raw - Q  written into the enriched rows of Y
template <typename T>
__global__ void k_enr_final(int n_enr, int N, const double *Yraw, const double *Q, T *Ye, int ld) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n_enr * N) return;
    int k = (int)(idx / N), j = (int)(idx % N);
    Ye[(long long)k * ld + j] = (T)(Yraw[idx] - (Q ? Q[idx] : 0.0));
}

template <typename A, typename B>
__global__ void k_cast(long long n, const A *x, B *y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (B)x[i];
}

// X' = Y_c - C^T Y_e rounded to bf16 with row stride ldb (padding columns and
// boundary rows zero): the B operand of the tensor-core cell products.
__global__ void k_xprime_bf16(MeshDev m, long long n_nodes, const float *Y, int N, int ldb,
                              const long long *node_ptr, const int *node_ent, const int *ent_atom,
                              const double *C, int use_c, __nv_bfloat16 *Xb) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n_nodes * ldb) return;
    long long n = idx / ldb;
    int j = (int)(idx % ldb);
    int ix = (int)(n % m.Gx), iy = (int)((n / m.Gx) % m.Gy), iz = (int)(n / ((long long)m.Gx * m.Gy));
    float out = 0.f;
    if (j < N && node_interior(m, ix, iy, iz)) {
        double v = (double)Y[n * N + j];
        if (use_c) {
            const float *Ye = Y + n_nodes * N;
            for (long long e = node_ptr[n]; e < node_ptr[n + 1]; ++e) {
                int g = node_ent[e];
                int I = ent_atom[g];
                const double *c = C + 4 * (long long)g;
                v -= c[0] * (double)Ye[(4 * I + 0) * (long long)N + j] + c[1] * (double)Ye[(4 * I + 1) * (long long)N + j] +
                     c[2] * (double)Ye[(4 * I + 2) * (long long)N + j] + c[3] * (double)Ye[(4 * I + 3) * (long long)N + j];
            }
        }
        out = (float)v;
    }
    Xb[idx] = __float2bfloat16_rn(out);
}

// HY_c[n] = sum over the cells containing node n of their per-cell product
// rows, plus the node-side coupling (H^ca X_e + P_c^T W).  Boundary rows 0.
__global__ void k_gather(MeshDev m, long long n_nodes, int N, const float *Yc, int ldy,
                         const long long *node_ptr, const int *node_ent, const int *ent_atom, const double *Hca,
                         const double *Pc, const float *Xe, const double *W, int use_h, int use_p, float *HY) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n_nodes * N) return;
    long long n = idx / N;
    int j = (int)(idx % N);
    int ix = (int)(n % m.Gx), iy = (int)((n / m.Gx) % m.Gy), iz = (int)(n / ((long long)m.Gx * m.Gy));
    if (!node_interior(m, ix, iy, iz)) { HY[idx] = 0.f; return; }
    int cxv[2], axv[2], cyv[2], ayv[2], czv[2], azv[2];
    int nxc = 0, nyc = 0, nzc = 0;
    auto split = [&](int i, int ncell, int *cv, int *av, int &cnt) {
        int q = i / m.p, r = i % m.p;
        if (r == 0) {
            if (q - 1 >= 0) { cv[cnt] = q - 1; av[cnt] = m.p; ++cnt; }
            if (q < ncell) { cv[cnt] = q; av[cnt] = 0; ++cnt; }
        } else {
            cv[cnt] = q; av[cnt] = r; ++cnt;
        }
    };
    split(ix, m.nx, cxv, axv, nxc);
    split(iy, m.ny, cyv, ayv, nyc);
    split(iz, m.nz, czv, azv, nzc);
    double acc = 0.0;
    for (int a = 0; a < nzc; ++a)
        for (int b = 0; b < nyc; ++b)
            for (int c = 0; c < nxc; ++c) {
                long long cell = ((long long)czv[a] * m.ny + cyv[b]) * m.nx + cxv[c];
                int l = (azv[a] * m.np1 + ayv[b]) * m.np1 + axv[c];
                acc += (double)Yc[(cell * m.ne + l) * ldy + j];
            }
    if (node_ptr) {
        for (long long e = node_ptr[n]; e < node_ptr[n + 1]; ++e) {
            int g = node_ent[e];
            int I = ent_atom[g];
            if (use_h) {
                const double *h = Hca + 4 * (long long)g;
                for (int f = 0; f < 4; ++f) acc += h[f] * (double)Xe[(long long)(4 * I + f) * N + j];
            }
            if (use_p) {
                const double *pc = Pc + 4 * (long long)g;
                for (int f = 0; f < 4; ++f) acc += pc[f] * W[(long long)(4 * I + f) * N + j];
            }
        }
    }
    HY[idx] = (float)acc;
}

// ---------------------------------------------------------------------------
// Row kernels of the tensor-core filter: one warp per FE node row (node
// coordinates and coupling lists are read once per row, lanes run over the
// columns).  All arithmetic is FP32; the values feed bf16 products.
// ---------------------------------------------------------------------------
__global__ void k_to_float_strided(long long rows, int N, const double *x, float *y, int ldy,
                                   __nv_bfloat16 *y16 = nullptr) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * N) return;
    const size_t o = (size_t)(idx / N) * ldy + idx % N;
    y[o] = (float)x[idx];
    if (y16) y16[o] = __float2bfloat16_rn((float)x[idx]);
}
// ---------------------------------------------------------------------------
// Vectorised row kernels of the tensor-core filter.  FE-row buffers use a row
// stride ldz = N rounded up to 4 floats (16-byte rows): lanes move float4s.
// ---------------------------------------------------------------------------
__device__ inline float4 f4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ inline float4 f4(const __nv_bfloat16 *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ inline void fma4(float4 &a, float s, const float4 b) {
    a.x += s * b.x; a.y += s * b.y; a.z += s * b.z; a.w += s * b.w;
}

// The two per-node kernels of the bf16 filter.  A warp takes a run of kRun
// consecutive nodes along x (same iy, iz), so the y/z part of the cell
// indexing is formed once per warp, and walks the run's rows as one flat list
// of float4 column groups (lane l takes groups l, l + 32, ...), so no lane
// idles when the row length is not a multiple of 128 floats.
constexpr int kRun = 8;

struct AxisCells {
    int k0, a0, two;   // the node lies in cell k0 at local index a0 (and in k0 + 1 at 0 if two)
};
__device__ __forceinline__ AxisCells axis_cells(int i, int p, int nc) {
    const int q = i / p, r = i - q * p;
    AxisCells a;
    if (r != 0) { a.k0 = q; a.a0 = r; a.two = 0; }
    else if (q > 0) { a.k0 = q - 1; a.a0 = p; a.two = q < nc ? 1 : 0; }
    else { a.k0 = q; a.a0 = 0; a.two = 0; }
    return a;
}

// bf16 quads: 4 consecutive columns as one 8-byte load/store
__device__ inline void st4(__nv_bfloat16 *p, const float4 v) {
    __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    uint2 pk;
    pk.x = *reinterpret_cast<uint32_t *>(&lo);
    pk.y = *reinterpret_cast<uint32_t *>(&hi);
    *reinterpret_cast<uint2 *>(p) = pk;
}

// One recurrence step of the bf16 filter at the FE nodes of a run, in the
// variables Y = M~^-1 Z (FE rows: Y = (M^cc)^-1 Z), stored in bf16:
//   HY[n] = sum over the cells of n of Y_cell[row(n)]
//   Y_k[n] = a ((M^cc_n)^-1 HY[n] - c Y_{k-1}[n]) - b Y_{k-2}[n] + a Ghat[n] ck
// (Eq. residualapprox multiplied by (M^cc)^-1, Ghat = (M^cc)^-1 G), all
// arithmetic in FP32.  The cell rows already hold the FE row's coupling
// E^T Y_e + P_c^T W (added by the cell products of the cell that owns the
// node), so this is a plain streaming pass.  The storage rounding of Y and
// Ghat is relative to residual-sized quantities, like the bf16 rounding of the
// cell operands (which are Y_{k-1} itself).  Cell rows: FP32 or bf16 (TC).
// A warp takes a run of kRun nodes along x and walks its rows as one flat
// list of 4-column groups (every lane busy; many independent loads in flight).
template <typename TC>
__global__ void __launch_bounds__(256, 4)
    k_gather_rec_b(MeshDev m, int nruns_x, int ldb, const TC *__restrict__ Yc, const double *__restrict__ minv,
                   const __nv_bfloat16 *__restrict__ Y1, const __nv_bfloat16 *__restrict__ Y0,
                   const __nv_bfloat16 *__restrict__ G, const float *__restrict__ ck, float a, float c, float b,
                   __nv_bfloat16 *__restrict__ Yn) {
    const int lane = threadIdx.x & 31;
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nrows = (long long)m.Gy * m.Gz;
    if (wid >= nrows * nruns_x) return;
    const int xr = (int)(wid % nruns_x);
    const long long yz = wid / nruns_x;
    const int iy = (int)(yz % m.Gy), iz = (int)(yz / m.Gy);
    const int x0 = xr * kRun;
    const int nrun = min(kRun, m.Gx - x0);
    const bool yz_in = iy > 0 && iz > 0 && iy < m.Gy - 1 && iz < m.Gz - 1;
    const long long n0 = yz * m.Gx + x0;
    int cyz[4];                // cell index without x (cells < 2^31)
    int lyz[4];
    bool vyz[4];
    {
        const AxisCells ay = axis_cells(iy, m.p, m.ny), az = axis_cells(iz, m.p, m.nz);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int sy = t & 1, sz = t >> 1;
            vyz[t] = (sy <= ay.two) && (sz <= az.two);
            const int cy = ay.k0 + sy, cz = az.k0 + sz;
            const int ly = sy ? 0 : ay.a0, lz = sz ? 0 : az.a0;
            cyz[t] = (cz * m.ny + cy) * m.nx;
            lyz[t] = (lz * m.np1 + ly) * m.np1;
        }
    }
    const int ncg = ldb / 4;
    int k = 0, cg = lane;
    while (cg >= ncg) { cg -= ncg; ++k; }
    for (; k < nrun;) {
        const int ix = x0 + k;
        const long long n = n0 + k;
        const int j = 4 * cg;
        const size_t row = (size_t)n * ldb + j;
        if (!(yz_in && ix > 0 && ix < m.Gx - 1)) {
            *reinterpret_cast<uint2 *>(Yn + row) = make_uint2(0u, 0u);
        } else {
            const AxisCells ax = axis_cells(ix, m.p, m.nx);
            float4 y[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int sx = u & 1, t = u >> 1;
                const bool ok = vyz[t] && (sx <= ax.two);
                const long long cell = (long long)(cyz[t] + ax.k0 + sx);
                const int l = lyz[t] + (sx ? 0 : ax.a0);
                y[u] = ok ? f4(Yc + (cell * m.ne + l) * ldb + j) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float4 y1 = f4(Y1 + row);
            const float4 y0 = Y0 ? f4(Y0 + row) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 gg = f4(G + row);
            const float4 kk = f4(ck + j);
            const float mi = (float)minv[n];
            // the cells in the order z, y, x (outer to inner)
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u) { acc.x += y[u].x; acc.y += y[u].y; acc.z += y[u].z; acc.w += y[u].w; }
            float4 yn;
            yn.x = a * (mi * acc.x - c * y1.x) - b * y0.x + a * gg.x * kk.x;
            yn.y = a * (mi * acc.y - c * y1.y) - b * y0.y + a * gg.y * kk.y;
            yn.z = a * (mi * acc.z - c * y1.z) - b * y0.z + a * gg.z * kk.z;
            yn.w = a * (mi * acc.w - c * y1.w) - b * y0.w + a * gg.w * kk.w;
            st4(Yn + row, yn);
        }
        cg += 32;
        while (cg >= ncg) { cg -= ncg; ++k; }
    }
}

// The bf16 node recurrence with 8-column groups (the filter's node pass for
// bf16 cell rows; the same arithmetic as k_gather_rec_b).  A warp takes a run
// of kRun nodes along x; it first lists, per node of the run, the rows of its
// up to 8 cells (z, y, x order; -1 where the node has no such cell, -2 for a
// Dirichlet node) and (M^cc_n)^-1 in shared memory, then walks the run's
// 16-byte column groups as one flat list, so the per-group work is the loads,
// the sum over the cells (in the listed order) and the recurrence, two columns
// per packed FP32 instruction.
__device__ __forceinline__ void bf8_to_f2(const uint4 v, float2 f[4]) {
    f[0] = make_float2(__uint_as_float(v.x << 16), __uint_as_float(v.x & 0xffff0000u));
    f[1] = make_float2(__uint_as_float(v.y << 16), __uint_as_float(v.y & 0xffff0000u));
    f[2] = make_float2(__uint_as_float(v.z << 16), __uint_as_float(v.z & 0xffff0000u));
    f[3] = make_float2(__uint_as_float(v.w << 16), __uint_as_float(v.w & 0xffff0000u));
}
__device__ __forceinline__ uint32_t f2_to_bf2(const float2 v) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __launch_bounds__(256, 4)
    k_gather_rec_c(MeshDev m, int nruns_x, int ldb, const __nv_bfloat16 *__restrict__ Yc,
                   const double *__restrict__ minv, const __nv_bfloat16 *__restrict__ Y1,
                   const __nv_bfloat16 *__restrict__ Y0, const __nv_bfloat16 *__restrict__ G,
                   const float *__restrict__ ck, float a, float c, float b, __nv_bfloat16 *__restrict__ Yn) {
    __shared__ int s_row[8][kRun][8];
    __shared__ float s_mi[8][kRun];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + w;
    const long long nrows = (long long)m.Gy * m.Gz;
    if (wid >= nrows * nruns_x) return;        // warp-uniform; no block-wide barrier below
    const int xr = (int)(wid % nruns_x);
    const long long yz = wid / nruns_x;
    const int iy = (int)(yz % m.Gy), iz = (int)(yz / m.Gy);
    const int x0 = xr * kRun;
    const int nrun = min(kRun, m.Gx - x0);
    const bool yz_in = iy > 0 && iz > 0 && iy < m.Gy - 1 && iz < m.Gz - 1;
    const long long n0 = yz * m.Gx + x0;
    {
        const AxisCells ay = axis_cells(iy, m.p, m.ny), az = axis_cells(iz, m.p, m.nz);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int e = lane + 32 * h, k = e >> 3, u = e & 7;
            const int ix = x0 + k;
            int row = -1;
            if (k < nrun) {
                if (!(yz_in && ix > 0 && ix < m.Gx - 1)) {
                    row = -2;
                } else {
                    const int sx = u & 1, sy = (u >> 1) & 1, sz = u >> 2;
                    const AxisCells ax = axis_cells(ix, m.p, m.nx);
                    if (sx <= ax.two && sy <= ay.two && sz <= az.two) {
                        const int cx = ax.k0 + sx, cy = ay.k0 + sy, cz = az.k0 + sz;
                        const int lx = sx ? 0 : ax.a0, ly = sy ? 0 : ay.a0, lz = sz ? 0 : az.a0;
                        row = ((cz * m.ny + cy) * m.nx + cx) * m.ne + (lz * m.np1 + ly) * m.np1 + lx;
                    }
                }
            }
            s_row[w][k][u] = row;
            if (u == 0 && k < nrun) s_mi[w][k] = (float)minv[n0 + k];
        }
    }
    __syncwarp();
    const int ncg = ldb / 8;
    const int total = nrun * ncg;
    int k = 0, cg = lane;
    while (cg >= ncg) { cg -= ncg; ++k; }
    const float2 a2 = make_float2(a, a), mc2 = make_float2(-c, -c), mb2 = make_float2(-b, -b);
    for (int item = lane; item < total; item += 32) {
        const long long n = n0 + k;
        const int j = 8 * cg;
        const size_t off = (size_t)n * ldb + j;
        const int4 r0 = *reinterpret_cast<const int4 *>(&s_row[w][k][0]);
        const int4 r1 = *reinterpret_cast<const int4 *>(&s_row[w][k][4]);
        if (r0.x == -2) {
            *reinterpret_cast<uint4 *>(Yn + off) = make_uint4(0u, 0u, 0u, 0u);
        } else {
            const int rows[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                v[u] = rows[u] >= 0 ? __ldg(reinterpret_cast<const uint4 *>(Yc + (size_t)rows[u] * ldb + j))
                                    : make_uint4(0u, 0u, 0u, 0u);
            const uint4 y1 = __ldg(reinterpret_cast<const uint4 *>(Y1 + off));
            const uint4 y0 = Y0 ? __ldg(reinterpret_cast<const uint4 *>(Y0 + off)) : make_uint4(0u, 0u, 0u, 0u);
            const uint4 gg = __ldg(reinterpret_cast<const uint4 *>(G + off));
            const float4 k0 = *reinterpret_cast<const float4 *>(ck + j), k1 = *reinterpret_cast<const float4 *>(ck + j + 4);
            float2 acc[4], f[4];
            bf8_to_f2(v[0], acc);
#pragma unroll
            for (int u = 1; u < 8; ++u) {
                bf8_to_f2(v[u], f);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = __fadd2_rn(acc[q], f[q]);
            }
            float2 f1[4], f0[4], fg[4];
            bf8_to_f2(y1, f1);
            bf8_to_f2(y0, f0);
            bf8_to_f2(gg, fg);
            const float2 kk[4] = {make_float2(k0.x, k0.y), make_float2(k0.z, k0.w), make_float2(k1.x, k1.y),
                                  make_float2(k1.z, k1.w)};
            const float mi = s_mi[w][k];
            const float2 mi2 = make_float2(mi, mi);
            uint4 o;
            uint32_t *op = &o.x;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                // a (mi HY - c Y1) - b Y0 + (a ck) Ghat
                const float2 t = __ffma2_rn(mi2, acc[q], __fmul2_rn(mc2, f1[q]));
                const float2 r = __ffma2_rn(a2, t, __fmul2_rn(mb2, f0[q]));
                op[q] = f2_to_bf2(__ffma2_rn(__fmul2_rn(a2, kk[q]), fg[q], r));
            }
            *reinterpret_cast<uint4 *>(Yn + off) = o;
        }
        cg += 32;
        while (cg >= ncg) { cg -= ncg; ++k; }
    }
}

// The coupling table of the cell products, YW[I][cb][r][c] (bf16, MN-major
// 8 x 8 core matrices): rows r < 4 are Y_e rows 4I + r, rows r >= 4 are W rows
// 4I + r - 4, column j = 8 cb + c; zero past N and for the extra block I = natoms.
__global__ void k_pack_yw(int natoms, int nCB, int N, int ldb, const __nv_bfloat16 *__restrict__ Ye16,
                          const __nv_bfloat16 *__restrict__ W16, __nv_bfloat16 *__restrict__ YW) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)(natoms + 1) * nCB * 64) return;
    const int cc = (int)(idx % 8), r = (int)((idx / 8) % 8);
    const long long ib = idx / 64;
    const int cb = (int)(ib % nCB), I = (int)(ib / nCB);
    const int j = 8 * cb + cc;
    __nv_bfloat16 v = __float2bfloat16_rn(0.f);
    if (I < natoms && j < N) {
        if (r < 4) {
            if (Ye16) v = Ye16[(size_t)(4 * I + r) * ldb + j];
        } else if (W16) {
            v = W16[(size_t)(4 * I + r - 4) * ldb + j];
        }
    }
    YW[idx] = v;
}

// Support reduction: warps over positions (8 rows in flight per warp), lanes
// over 4-column vectors (two 128-column slots), one block per (chunk, atom).
__device__ inline float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ inline float4 ld4(const __nv_bfloat16 *p) { return f4(p); }

template <typename T>
__global__ void __launch_bounds__(256, 4) k_support_reduce3(const long long *sup_off, const int *sup_node,
                                                         const float *coefA, const float *coefB, const T *S,
                                                         const double *scale, int N, int ld, int chunk, int nch,
                                                         const int2 *order, double *part) {
    // thread t: float4 column group cg = t % ncg, position lane pl = t / ncg
    __shared__ float acc[8][256];
    // block -> (atom, chunk): from the order table (blocks sorted by their first
    // node, so that atoms sharing a region read its rows while they are in L2)
    const int I = order ? order[blockIdx.x].x : blockIdx.y;
    const int ch = order ? order[blockIdx.x].y : blockIdx.x;
    const int ncg = (N + 3) / 4;                 // <= 64
    const int npl = blockDim.x / ncg;
    const int cg = threadIdx.x % ncg, pl = threadIdx.x / ncg;
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) acc[i / 256][i % 256] = 0.f;
    __syncthreads();
    const long long beg = sup_off[I] + (long long)ch * chunk;
    const long long end = min(sup_off[I + 1], beg + chunk);
    const bool two = coefB != nullptr;
    float4 r[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (pl < npl) {
        const int j = 4 * cg;
        for (long long g0 = beg + 4 * pl; g0 < end; g0 += 4 * npl) {
            int nodes[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) nodes[u] = (g0 + u < end) ? sup_node[g0 + u] : -1;
            float4 sv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sv[u] = nodes[u] >= 0 ? ld4(S + (long long)nodes[u] * ld + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                if (scale && nodes[u] >= 0) {
                    const float sc = (float)scale[nodes[u]];
                    sv[u].x *= sc; sv[u].y *= sc; sv[u].z *= sc; sv[u].w *= sc;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (nodes[u] < 0) continue;
                const float4 qa = ld4(coefA + 4 * (g0 + u));
                fma4(r[0], qa.x, sv[u]);
                fma4(r[1], qa.y, sv[u]);
                fma4(r[2], qa.z, sv[u]);
                fma4(r[3], qa.w, sv[u]);
                if (two) {
                    const float4 qb = ld4(coefB + 4 * (g0 + u));
                    fma4(r[4], qb.x, sv[u]);
                    fma4(r[5], qb.y, sv[u]);
                    fma4(r[6], qb.z, sv[u]);
                    fma4(r[7], qb.w, sv[u]);
                }
            }
        }
        const int nr = two ? 8 : 4;
        for (int i = 0; i < nr; ++i) {
            atomicAdd(&acc[i][j + 0], r[i].x);
            atomicAdd(&acc[i][j + 1], r[i].y);
            atomicAdd(&acc[i][j + 2], r[i].z);
            atomicAdd(&acc[i][j + 3], r[i].w);
        }
    }
    __syncthreads();
    const int nr = two ? 8 : 4;
    double *o = part + ((long long)(I * nch + ch) * 8) * N;
    for (int i = threadIdx.x; i < nr * 256; i += blockDim.x) {
        const int rr = i / 256, jj = i % 256;
        if (jj < N) o[(long long)rr * N + jj] = acc[rr][jj];
    }
}

// P_c Y_c over the compacted projector support lists, bf16 Y (the mixed
// filter's P-only reduction).  One block per (atom, chunk of kPChunk
// entries), from the order table; the chunk's node indices and P_c rows are
// staged in shared memory first, so the loop carries no dependent index
// load.  Thread t takes 8-column group t % ngr (16-byte loads) at position
// lane t / ngr and keeps 8 rows in flight; the position lanes are then
// summed in a fixed order (deterministic), rows 0-3 of the chunk's partials.
constexpr int kPChunk = 1024;
__global__ void __launch_bounds__(256, 3) k_psup_reduce(const long long *__restrict__ sup_off,
                                                       const int *__restrict__ sup_node,
                                                       const float4 *__restrict__ coef,
                                                       const __nv_bfloat16 *__restrict__ Y, int N, int ldb, int nch,
                                                       const int2 *__restrict__ order, double *__restrict__ part) {
    __shared__ int s_node[kPChunk];
    __shared__ float4 s_coef[kPChunk];
    const int I = order[blockIdx.x].x, ch = order[blockIdx.x].y;
    const long long beg = sup_off[I] + (long long)ch * kPChunk;
    const int cnt = (int)max(0LL, min(sup_off[I + 1] - beg, (long long)kPChunk));
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        s_node[i] = sup_node[beg + i];
        s_coef[i] = coef[beg + i];
    }
    __syncthreads();
    const int ngr = ldb / 8, npl = blockDim.x / ngr;      // ngr <= 32 (N <= 256)
    const int g = threadIdx.x % ngr, pl = threadIdx.x / ngr;
    float2 acc[4][4];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[f][c] = make_float2(0.f, 0.f);
    if (pl < npl) {
        const __nv_bfloat16 *Yg = Y + 8 * g;
        for (int i0 = pl; i0 < cnt; i0 += 8 * npl) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * npl;
                v[u] = i < cnt ? __ldg(reinterpret_cast<const uint4 *>(Yg + (size_t)s_node[i] * ldb))
                               : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * npl;
                if (i >= cnt) break;
                const float4 q = s_coef[i];
                float2 y[4];
                bf8_to_f2(v[u], y);
                const float2 qx = make_float2(q.x, q.x), qy = make_float2(q.y, q.y), qz = make_float2(q.z, q.z),
                             qw = make_float2(q.w, q.w);
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) {          // two columns per packed FMA
                    acc[0][c2] = __ffma2_rn(qx, y[c2], acc[0][c2]);
                    acc[1][c2] = __ffma2_rn(qy, y[c2], acc[1][c2]);
                    acc[2][c2] = __ffma2_rn(qz, y[c2], acc[2][c2]);
                    acc[3][c2] = __ffma2_rn(qw, y[c2], acc[3][c2]);
                }
            }
        }
    }
    // two halves (f = 0, 1 then 2, 3): [npl][2][ldb] floats = 16 npl ngr <= 4096 fit in s_coef
    float *red = reinterpret_cast<float *>(s_coef);
    double *o = part + ((long long)I * nch + ch) * 8 * N;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        __syncthreads();                                  // s_coef (or the previous half) is free
        if (pl < npl)
#pragma unroll
            for (int f = 0; f < 2; ++f)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    red[((size_t)pl * 2 + f) * ldb + 8 * g + 2 * c] = acc[2 * h2 + f][c].x;
                    red[((size_t)pl * 2 + f) * ldb + 8 * g + 2 * c + 1] = acc[2 * h2 + f][c].y;
                }
        __syncthreads();
        for (int t = threadIdx.x; t < 2 * N; t += blockDim.x) {
            const int f = t / N, j = t - f * N;
            float sum = 0.f;
            for (int l = 0; l < npl; ++l) sum += red[((size_t)l * 2 + f) * ldb + j];
            o[(long long)(2 * h2 + f) * N + j] = sum;
        }
    }
}

// Start of the bf16 filter, a warp per row, lanes over 4-column groups.
// g = HV - (M V) diag(lv): the eigen-residual G (the standard filter passes
// lv = c and the approximate M~; both are diagonal M^cc on the FE rows, formed
// here from V, so M V is never stored for them; MVe holds the enriched rows
// of M V).  FE rows (the Y = (M^cc)^-1 Z variables, bf16, row stride ldb,
// zero at the Dirichlet nodes and in the padding columns): Ghat = (M^cc)^-1 g,
// Y_1 = s1e Ghat, Y_0 = V (standard filter only).  Enriched rows (FP32,
// stride ldb): G_e = g, Z_1 = s1e g, Z_0 = MVe (standard only).
__global__ void __launch_bounds__(256) k_filter_start_b(long long nn, long long rows, int N, int ldb,
                                                        const double *__restrict__ HV, const double *__restrict__ V,
                                                        const double *__restrict__ MVe,
                                                        const double *__restrict__ lv, const double *__restrict__ mcc,
                                                        const double *__restrict__ minv, double s1e,
                                                        __nv_bfloat16 *__restrict__ Gb,
                                                        __nv_bfloat16 *__restrict__ Y1b,
                                                        __nv_bfloat16 *__restrict__ Y0b, float *__restrict__ Ge,
                                                        float *__restrict__ Z1e, float *__restrict__ Z0e) {
    // lv split once per block (N <= 256 on this path)
    __shared__ float2 s_lv[256];
    for (int j = threadIdx.x; j < N && j < 256; j += blockDim.x) {
        float h, l;
        f64_split(lv[j], h, l);
        s_lv[j] = make_float2(h, l);
    }
    __syncthreads();
    const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    const bool fe = r < nn;
    const double mi = fe ? minv[r] : 0.0;
    float mih, mil;
    f64_split(mi, mih, mil);
    const bool mi_nz = mi != 0.0;
    const double *hv = HV + r * N, *vv = V + r * N;
    const double *mv = fe ? nullptr : MVe + (r - nn) * N;
    for (int j0 = 4 * (threadIdx.x & 31); j0 < ldb; j0 += 128) {
        float g[4], v[4], m4[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int j = j0 + i;
            g[i] = v[i] = m4[i] = 0.f;
            if (j < N) {
                if (fe) {
                    // (M^cc)^-1 (HV - M^cc V lv) = (M^cc)^-1 HV - lv V in double-single
                    // arithmetic on the FP32 pipe (operands split by integer operations;
                    // zero at the Dirichlet nodes)
                    if (mi_nz) {
                        float hh, hl, vh, vl;
                        f64_split(hv[j], hh, hl);
                        f64_split(vv[j], vh, vl);
                        const float2 l2 = s_lv[j];
                        g[i] = ds_mul_sub(mih, mil, hh, hl, l2.x, l2.y, vh, vl);
                        if (Y0b) v[i] = vh;
                    }
                } else {
                    const double mvj = mv[j];
                    g[i] = (float)(hv[j] - mvj * lv[j]);
                    m4[i] = (float)mvj;
                }
            }
        }
        const float4 G4 = make_float4(g[0], g[1], g[2], g[3]);
        const float4 S4 = make_float4((float)s1e * g[0], (float)s1e * g[1], (float)s1e * g[2], (float)s1e * g[3]);
        if (fe) {
            const size_t o = (size_t)r * ldb + j0;
            st4(Gb + o, G4);
            st4(Y1b + o, S4);
            if (Y0b) st4(Y0b + o, make_float4(v[0], v[1], v[2], v[3]));
        } else {
            const size_t o = (size_t)(r - nn) * ldb + j0;
            *reinterpret_cast<float4 *>(Ge + o) = G4;
            *reinterpret_cast<float4 *>(Z1e + o) = S4;
            if (Z0e) *reinterpret_cast<float4 *>(Z0e + o) = make_float4(m4[0], m4[1], m4[2], m4[3]);
        }
    }
}

__global__ void k_enr_minv_f(int n_enr, int N, int ld, const double *Binv, const float *X, float *Y, int ldy,
                             __nv_bfloat16 *Y16 = nullptr) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_enr * N) return;
    const int k = idx / N, j = idx % N;
    const int I = k / 4, f = k % 4;
    const double *bb = Binv + 16 * I + 4 * f;
    float s = 0.f;
    for (int g = 0; g < 4; ++g) s += (float)bb[g] * X[(size_t)(4 * I + g) * ld + j];
    Y[(size_t)k * ldy + j] = s;
    if (Y16) Y16[(size_t)k * ldy + j] = __float2bfloat16_rn(s);
}
__global__ void k_enr_rec_v(int n_enr, int N, int ldz, const double *Yraw, const double *Q, const float *Z1,
                            const float *Z0, const float *G, const float *ck, float a, float c, float b, float *Zn) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_enr * ldz) return;
    const int k = idx / ldz, j = idx % ldz;
    const size_t o = (size_t)k * ldz + j;
    if (j >= N) { Zn[o] = 0.f; return; }
    const float hy = (float)(Yraw[(size_t)k * N + j] - (Q ? Q[(size_t)k * N + j] : 0.0));
    const float z0 = Z0 ? Z0[o] : 0.f;
    Zn[o] = a * (hy - c * Z1[o]) - b * z0 + a * G[o] * ck[j];
}
// V_out = M~^-1 Z_m + V diag(C_m(lam)): FE rows from the bf16 Y_m, enriched
// rows from Ye = (M~^ee)^-1 Z_e (FP32); warp per row.
__global__ void __launch_bounds__(256) k_vout_b(long long nn, long long rows, int N, int ldb,
                                                const __nv_bfloat16 *__restrict__ Yb, const float *__restrict__ Ye,
                                                const double *__restrict__ V, const double *__restrict__ cm,
                                                double *__restrict__ Vout) {
    const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    const bool fe = r < nn;
    for (int j = threadIdx.x & 31; j < N; j += 32) {
        const float y = fe ? __bfloat162float(Yb[r * ldb + j]) : Ye[(r - nn) * ldb + j];
        Vout[r * N + j] = (double)y + V[r * N + j] * cm[j];
    }
}

// Row-parallel elementwise helpers (warp per row, no 64-bit division)
template <typename T>
__global__ void __launch_bounds__(256) k_rows_residual(long long rows, int N, const double *HV, const double *MV,
                                                       const double *lam, T *G) {
    const long long r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (r >= rows) return;
    for (int j = threadIdx.x & 31; j < N; j += 32) G[r * N + j] = (T)(HV[r * N + j] - MV[r * N + j] * lam[j]);
}

// zero the Dirichlet boundary rows of a block (they are not unknowns)
__global__ void k_zero_boundary(MeshDev m, long long n_nodes, int N, double *X) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n_nodes * N) return;
    long long n = idx / N;
    int ix = (int)(n % m.Gx), iy = (int)((n / m.Gx) % m.Gy), iz = (int)(n / ((long long)m.Gx * m.Gy));
    if (!node_interior(m, ix, iy, iz)) X[idx] = 0.0;
}

// ---- M^E, (M~^E)^-1 ------------------------------------------------------
template <typename T>
__global__ void k_diag_scale(long long n, int N, const double *d, const T *X, T *Y) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n * N) return;
    Y[idx] = (T)(d[idx / N] * (double)X[idx]);
}
// enriched rows: Y_e = A X_e with A dense (n_enr x n_enr) or atom blocks (4x4)
template <typename T>
__global__ void k_enr_mat(int n_enr, int N, const double *A, int blocks, const T *X, T *Y) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n_enr * N) return;
    int k = (int)(idx / N), j = (int)(idx % N);
    double s = 0.0;
    if (blocks) {
        int I = k / 4, f = k % 4;
        const double *b = A + 16 * I + 4 * f;
        for (int g = 0; g < 4; ++g) s += b[g] * (double)X[(long long)(4 * I + g) * N + j];
    } else {
        for (int g = 0; g < n_enr; ++g) s += A[(long long)k * n_enr + g] * (double)X[(long long)g * N + j];
    }
    Y[idx] = (T)s;
}

// ---- residual Chebyshev recurrence ----------------------------------------
// G = HV - MV diag(lam)
__global__ void k_eig_residual(long long rows, int N, const double *HV, const double *MV, const double *lam,
                               double *G) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * N) return;
    G[idx] = HV[idx] - MV[idx] * lam[idx % N];
}
// Z_k = a (HY - c Z1) - b Z0 + a G ck   (a = 2 s_k / e, b = s_{k-1} s_k)
template <typename T>
__global__ void k_recurrence(long long n, int N, double a, double c, double b, const T *HY, const T *Z1,
                             const T *Z0, const double *G, const double *ck, T *Zn) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n) return;
    double z0 = Z0 ? (double)Z0[idx] : 0.0;
    double v = a * ((double)HY[idx] - c * (double)Z1[idx]) - b * z0 + a * G[idx] * ck[idx % N];
    Zn[idx] = (T)v;
}
template <typename T>
__global__ void k_scale_to(long long n, double s, const double *G, T *Z) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < n) Z[idx] = (T)(s * G[idx]);
}
// Standard filter start, written in the residual variables Z = M~ Y:
// Z_0 = M~ V, Z_1 = (s1/e)(H V - c M~ V); G holds H V - c M~ V
template <typename T>
__global__ void k_std_start(long long n, double c, double s1e, const double *HV, const double *MtV, double *G,
                            T *Z0, T *Z1) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const double g = HV[idx] - c * MtV[idx];
    G[idx] = g;
    Z0[idx] = (T)MtV[idx];
    Z1[idx] = (T)(s1e * g);
}
// Vout = Y + V diag(cm)   (Y = M~^-1 Z_m)
template <typename T>
__global__ void k_vout(long long n, int N, const T *Y, const double *V, const double *cm, double *Vout) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < n) Vout[idx] = (double)Y[idx] + V[idx] * cm[idx % N];
}

// ---- Rayleigh-Ritz ----------------------------------------------------------
// Partial Gram blocks: part[chunk][i][j] = sum_{r in chunk} A[r][i] B[r][j]
__global__ void k_gram_partial(long long rows, int N, const double *A, const double *B, long long chunk,
                               double *part) {
    __shared__ double sA[32][33], sB[32][33];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.z * 32;
    const long long r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 256 threads: ty 0..7
    double acc[4] = {0, 0, 0, 0};
    for (long long rb = r0; rb < r1; rb += 32) {
        for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
            int rr = t / 32, cc = t % 32;
            long long r = rb + rr;
            sA[rr][cc] = (r < r1 && i0 + cc < N) ? A[r * N + i0 + cc] : 0.0;
            sB[rr][cc] = (r < r1 && j0 + cc < N) ? B[r * N + j0 + cc] : 0.0;
        }
        __syncthreads();
        for (int rr = 0; rr < 32; ++rr) {
            double bv = sB[rr][tx];
            for (int q = 0; q < 4; ++q) acc[q] += sA[rr][ty + 8 * q] * bv;
        }
        __syncthreads();
    }
    double *o = part + (long long)blockIdx.x * N * N;
    for (int q = 0; q < 4; ++q) {
        int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < N && j < N) o[(long long)i * N + j] = acc[q];
    }
}
__global__ void k_gram_sum(int N, int nch, const double *part, double *out) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)N * N) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(long long)c * N * N + idx];
    out[idx] = s;
}
// symmetrise and scale (Jacobi): out_ij = (A_ij + A_ji)/2 / (d_i d_j), d_i = sqrt(S_ii)
__global__ void k_rr_scale(int N, const double *S0, const double *H0, double *Ss, double *Hs, double *d) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)N * N) return;
    int i = (int)(idx / N), j = (int)(idx % N);
    double di = sqrt(S0[(long long)i * N + i]), dj = sqrt(S0[(long long)j * N + j]);
    if (i == j) d[i] = di;
    Hs[idx] = 0.5 * (H0[(long long)i * N + j] + H0[(long long)j * N + i]) / (di * dj);
    Ss[idx] = 0.5 * (S0[(long long)i * N + j] + S0[(long long)j * N + i]) / (di * dj);
}
// Q (row-major) = D^-1 Qcol  : Qr[i][j] = Qc[i + j N] / d_i
__global__ void k_rr_unscale(int N, const double *Qc, const double *d, double *Qr) {
    long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)N * N) return;
    int i = (int)(idx / N), j = (int)(idx % N);
    Qr[idx] = Qc[i + (long long)j * N] / d[i];
}
// out = in Q (rows x N) with Q row-major N x N
__global__ void k_rotate(long long rows, int N, const double *in, const double *Q, double *out) {
    extern __shared__ double sR[];   // 16 rows x N
    const long long r0 = blockIdx.x * 16LL;
    for (int t = threadIdx.x; t < 16 * N; t += blockDim.x) {
        long long r = r0 + t / N;
        sR[t] = r < rows ? in[r * N + (t % N)] : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 16 * N; t += blockDim.x) {
        int rr = t / N, j = t % N;
        long long r = r0 + rr;
        if (r >= rows) continue;
        double s = 0.0;
        for (int i = 0; i < N; ++i) s += sR[rr * N + i] * Q[(long long)i * N + j];
        out[r * N + j] = s;
    }
}
// column sums of squares of R = HX - MX diag(lam), partial per block
__global__ void k_resid_partial(long long rows, int N, const double *HX, const double *MX, const double *lam,
                                long long chunk, double *part) {
    const long long r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double s = 0.0;
        for (long long r = r0; r < r1; ++r) {
            double v = HX[r * N + j] - MX[r * N + j] * lam[j];
            s += v * v;
        }
        part[(long long)blockIdx.x * N + j] = s;
    }
}
__global__ void k_colsum(int N, int nch, const double *part, double *out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[(long long)c * N + j];
    out[j] = s;
}
// dot products of single vectors: partial sums
__global__ void k_dot_partial(long long n, const double *a, const double *b, double *part) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}
__global__ void k_axpby3(long long n, double a, const double *x, double b, const double *y, double c,
                         const double *z, double *out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i] + (z ? c * z[i] : 0.0);
}

// host: eigenvalues/vectors of a small symmetric matrix by cyclic Jacobi
void jacobi_eig(int n, std::vector<double> A, std::vector<double> &w, std::vector<double> &V) {
    V.assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
        if (off < 1e-30) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double th = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

// Chebyshev scalars C_k(lam_j), k = 0..m (Eq. ChebyRecur), table (m+1) x N
void cheb_table(int m, int N, const double *lam, double a, double b, double a0, std::vector<double> &ck,
                std::vector<double> &sig) {
    const double e = 0.5 * (b - a), c = 0.5 * (b + a), s1 = e / (a0 - c);
    ck.assign((size_t)(m + 1) * N, 0.0);
    sig.assign(m + 1, 0.0);
    sig[1] = s1;
    for (int j = 0; j < N; ++j) {
        ck[j] = 1.0;
        if (m >= 1) ck[N + j] = s1 * (lam[j] - c) / e;
    }
    double sp = s1;
    for (int k = 2; k <= m; ++k) {
        double s = 1.0 / (2.0 / s1 - sp);
        sig[k] = s;
        for (int j = 0; j < N; ++j)
            ck[(size_t)k * N + j] = (2.0 * s / e) * (lam[j] - c) * ck[(size_t)(k - 1) * N + j] -
                                    sp * s * ck[(size_t)(k - 2) * N + j];
        sp = s;
    }
}

}  // namespace

// ===========================================================================
// infrastructure
// ===========================================================================
efe_status efe_check_launch(efe_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ctx->err = std::string(what) + ": " + cudaGetErrorString(e);
        return EFE_ERR_CUDA;
    }
    return EFE_OK;
}
efe_status efe_alloc(efe_ctx *ctx, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        return EFE_ERR_OOM;
    }
    return EFE_OK;
}
efe_status efe_workspace(efe_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return EFE_OK;
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->d_ws) cudaFree(ctx->d_ws);
    ctx->d_ws = nullptr;
    ctx->ws_bytes = 0;
    EFE_TRY(efe_alloc(ctx, &ctx->d_ws, bytes));
    ctx->ws_bytes = bytes;
    return EFE_OK;
}
efe_status efe_partials(efe_ctx *ctx, size_t doubles) {
    if (doubles * 8 <= ctx->part_bytes) return EFE_OK;
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->d_part) cudaFree(ctx->d_part);
    ctx->d_part = nullptr;
    ctx->part_bytes = 0;
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_part, doubles * 8));
    ctx->part_bytes = doubles * 8;
    return EFE_OK;
}
efe_status efe_pinned(efe_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->pinned_bytes) return EFE_OK;
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->h_pinned = nullptr;
    ctx->pinned_bytes = 0;
    EFE_CUDA(ctx, cudaMallocHost((void **)&ctx->h_pinned, bytes));
    ctx->pinned_bytes = bytes;
    return EFE_OK;
}

namespace {

// Scratch layout for one H^E product on N columns (doubles):
//   Xp  n_nodes*N | part 64*natoms*8*N | Rh n_enr*N | Wc n_proj*N | W n_proj*N | Yraw n_enr*N | Q n_enr*N
struct HxScratch {
    double *part, *Rh, *Wc, *W, *Yraw, *Q;
    int nch, chunk;
};

efe_status hx_scratch(efe_ctx *ctx, int N, HxScratch &s) {
    long long maxsup = 0;
    for (int I = 0; I < ctx->natoms; ++I) maxsup = std::max(maxsup, ctx->sup_off[I + 1] - ctx->sup_off[I]);
    s.chunk = 1024;
    s.nch = (int)std::max<long long>(1, (maxsup + s.chunk - 1) / s.chunk);
    // partial sums: 8 rows per (atom, chunk)
    const size_t npart = (size_t)s.nch * std::max(ctx->natoms, 1) * 8 * N;
    size_t need = npart + (size_t)(3 * ctx->n_enr + 2 * ctx->n_proj) * N + 64;
    EFE_TRY(efe_partials(ctx, need));
    double *p = ctx->d_part;
    s.part = p;
    p += npart;
    s.Rh = p; p += (size_t)ctx->n_enr * N;
    s.Wc = p; p += (size_t)ctx->n_proj * N;
    s.W = p; p += (size_t)ctx->n_proj * N;
    s.Yraw = p; p += (size_t)ctx->n_enr * N;
    s.Q = p;
    return EFE_OK;
}

// Launch order of the support reductions: every (atom, chunk) pair, sorted by
// the chunk's first support node (chunks past an atom's list keep their slot:
// their blocks write the zero partials the sum reads).  off/d_nodes: the
// per-atom lists (all support entries, or those with a projector row).
efe_status build_chunk_order(efe_ctx *ctx, const std::vector<long long> &off, const int *d_nodes, int chunk,
                             int nch, int2 **out) {
    const int na = std::max(ctx->natoms, 1);
    const long long total = off.empty() ? 0 : off.back();
    std::vector<int> first((size_t)std::max(total, 1LL));
    if (total > 0) EFE_CUDA(ctx, cudaMemcpy(first.data(), d_nodes, sizeof(int) * total, cudaMemcpyDeviceToHost));
    std::vector<std::pair<long long, int2>> key;
    key.reserve((size_t)na * nch);
    for (int I = 0; I < ctx->natoms; ++I)
        for (int c = 0; c < nch; ++c) {
            const long long g = off[I] + (long long)c * chunk;
            const long long k = g < off[I + 1] ? (long long)first[g] : (1LL << 62);
            key.push_back({k, make_int2(I, c)});
        }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<long long, int2> &a, const std::pair<long long, int2> &b) {
                         return a.first < b.first;
                     });
    std::vector<int2> ord(key.size());
    for (size_t i = 0; i < key.size(); ++i) ord[i] = key[i].second;
    if (*out) cudaFree(*out);
    *out = nullptr;
    EFE_TRY(efe_alloc(ctx, (void **)out, sizeof(int2) * std::max<size_t>(ord.size(), 1)));
    if (!ord.empty()) EFE_CUDA(ctx, cudaMemcpy(*out, ord.data(), sizeof(int2) * ord.size(), cudaMemcpyHostToDevice));
    return EFE_OK;
}

efe_status chunk_order(efe_ctx *ctx, int chunk, int nch) {
    if (ctx->d_chunk_order && ctx->chunk_order_nch == nch) return EFE_OK;
    EFE_TRY(build_chunk_order(ctx, ctx->sup_off, ctx->d_sup_node, chunk, nch, &ctx->d_chunk_order));
    ctx->chunk_order_nch = nch;
    return EFE_OK;
}

// The support entries with a nonzero projector row (P_c vanishes outside the
// projector ball, while the supports also cover the enrichment's one-cell
// dilation), per atom in node order, with their P_c rows; built once.
efe_status p_support_lists(efe_ctx *ctx, int chunk, int *nch) {
    if (!ctx->d_psup_off) {
        const long long S = ctx->sup_total;
        std::vector<int> node((size_t)std::max(S, 1LL));
        std::vector<float> pc((size_t)std::max(4 * S, 4LL));
        if (S > 0) {
            EFE_CUDA(ctx, cudaMemcpy(node.data(), ctx->d_sup_node, sizeof(int) * S, cudaMemcpyDeviceToHost));
            EFE_CUDA(ctx, cudaMemcpy(pc.data(), ctx->d_Pc32, sizeof(float) * 4 * S, cudaMemcpyDeviceToHost));
        }
        std::vector<long long> off(ctx->natoms + 1, 0);
        std::vector<int> pn;
        std::vector<float> pv;
        for (int I = 0; I < ctx->natoms; ++I) {
            for (long long g = ctx->sup_off[I]; g < ctx->sup_off[I + 1]; ++g) {
                const float *q = &pc[4 * g];
                if (q[0] == 0.f && q[1] == 0.f && q[2] == 0.f && q[3] == 0.f) continue;
                pn.push_back(node[g]);
                pv.insert(pv.end(), q, q + 4);
            }
            off[I + 1] = (long long)pn.size();
        }
        if (pn.empty()) {
            pn.push_back(0);
            pv.assign(4, 0.f);
        }
        ctx->psup_off = off;
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_psup_off, sizeof(long long) * off.size()));
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_psup_node, sizeof(int) * pn.size()));
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_psup_coef, sizeof(float) * pv.size()));
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_psup_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice));
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_psup_node, pn.data(), sizeof(int) * pn.size(), cudaMemcpyHostToDevice));
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_psup_coef, pv.data(), sizeof(float) * pv.size(), cudaMemcpyHostToDevice));
    }
    long long maxs = 0;
    for (int I = 0; I < ctx->natoms; ++I) maxs = std::max(maxs, ctx->psup_off[I + 1] - ctx->psup_off[I]);
    *nch = (int)std::max<long long>(1, (maxs + chunk - 1) / chunk);
    if (!ctx->d_pchunk_order || ctx->pchunk_nch != *nch) {
        EFE_TRY(build_chunk_order(ctx, ctx->psup_off, ctx->d_psup_node, chunk, *nch, &ctx->d_pchunk_order));
        ctx->pchunk_nch = *nch;
    }
    return EFE_OK;
}

}  // namespace

// Generic H^E product for storage type T (double or float).  Xp: n_nodes x N scratch.
template <typename T>
static efe_status hx_generic(efe_ctx *ctx, const T *X, T *Y, int N, const T *He, T *Xp) {
    const MeshDev &m = ctx->m;
    const long long nn = ctx->n_nodes;
    const int ld = N;
    const bool cpl = (ctx->enrich || ctx->nonlocal) && ctx->natoms > 0;
    HxScratch s{};
    if (cpl) EFE_TRY(hx_scratch(ctx, N, s));
    // (1) X' = T X (FE part)
    k_xprime<T><<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(m, nn, X, Xp, N, ld, ctx->d_node_ptr, ctx->d_node_ent,
                                                            ctx->d_ent_atom, ctx->d_C, ctx->enrich ? 1 : 0);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_xprime"));
    // (2) cell products
    EFE_CUDA(ctx, cudaMemsetAsync(Y, 0, sizeof(T) * ctx->n_rows * N, ctx->stream));
    EFE_TRY(launch_cells<T>(ctx, He, (long long)m.ne * m.ne, Xp, Y, N, ld));
    if (!cpl) return EFE_OK;
    const T *Xe = X + nn * ld;
    const long long *d_so = ctx->d_sup_off;
    dim3 gr(s.nch, ctx->natoms);
    // (3) R = [Hca; Pc] X'  (support reductions)
    k_support_reduce<T><<<gr, 128, 0, ctx->stream>>>(d_so, ctx->d_sup_node, ctx->enrich ? ctx->d_Hca : ctx->d_Pc,
                                                     (ctx->enrich && ctx->nonlocal) ? ctx->d_Pc : nullptr, Xp, N, ld,
                                                     s.chunk, s.nch, s.part);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_support_reduce"));
    {
        long long n = (long long)ctx->natoms * 8 * N;
        double *oA = ctx->enrich ? s.Rh : s.Wc;
        double *oB = (ctx->enrich && ctx->nonlocal) ? s.Wc : nullptr;
        k_support_sum<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->natoms, s.nch, N, s.part, oA, oB);
        ctx->launches++;
    }
    // (4) W and the raw enriched rows
    if (ctx->nonlocal) {
        k_proj_w<T><<<nblk((long long)ctx->n_proj * N, 256), 256, 0, ctx->stream>>>(
            ctx->n_proj, ctx->n_enr, s.Wc, ctx->enrich ? ctx->d_Pa : nullptr, Xe, ld, ctx->d_hproj, N, s.W);
        ctx->launches++;
    }
    if (ctx->enrich) {
        k_enr_raw<T><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(
            ctx->n_enr, ctx->n_proj, s.Rh, ctx->d_Haa, ctx->nonlocal ? ctx->d_Pa : nullptr, s.W, Xe, ld, N, s.Yraw);
        ctx->launches++;
    }
    // (5) node-side coupling into Y_c
    k_node_coupling<T><<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(nn, ctx->d_node_ptr, ctx->d_node_ent,
                                                                   ctx->d_ent_atom, ctx->d_Hca, ctx->d_Pc, Xe, ld, s.W,
                                                                   N, Y, ctx->enrich ? 1 : 0, ctx->nonlocal ? 1 : 0);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_node_coupling"));
    if (!ctx->enrich) return EFE_OK;
    // (6) Q = C Y_c and (7) Y_e = Y_e,raw - Q
    k_support_reduce<T><<<gr, 128, 0, ctx->stream>>>(d_so, ctx->d_sup_node, ctx->d_C, nullptr, Y, N, ld, s.chunk,
                                                     s.nch, s.part);
    {
        long long n = (long long)ctx->natoms * 8 * N;
        k_support_sum<<<nblk(n, 256), 256, 0, ctx->stream>>>(ctx->natoms, s.nch, N, s.part, s.Q, nullptr);
    }
    k_enr_final<T><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(ctx->n_enr, N, s.Yraw, s.Q,
                                                                                   Y + nn * ld, ld);
    ctx->launches += 3;
    return efe_check_launch(ctx, "k_enr_final");
}


// H^E Y with the cell products on tcgen05 tensor cores (bf16 operands, FP32
// accumulate); Y, HY: float rows x N.  Scratch: Xb (bf16 n_nodes x ldb) and
// Ycells (float n_cells x ne x ldy).
static efe_status hx_bf16(efe_ctx *ctx, const float *Y, float *HY, int N, __nv_bfloat16 *Xb, float *Ycells) {
    const MeshDev &m = ctx->m;
    const long long nn = ctx->n_nodes;
    const int ldb = (N + 7) / 8 * 8, ldy = (N + 3) / 4 * 4;
    const bool cpl = (ctx->enrich || ctx->nonlocal) && ctx->natoms > 0;
    HxScratch s{};
    if (cpl) EFE_TRY(hx_scratch(ctx, N, s));
    k_xprime_bf16<<<nblk(nn * ldb, 256), 256, 0, ctx->stream>>>(m, nn, Y, N, ldb, ctx->d_node_ptr, ctx->d_node_ent,
                                                               ctx->d_ent_atom, ctx->d_C, ctx->enrich ? 1 : 0, Xb);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_xprime_bf16"));
    {
        auto *ev = cell_event_pair(ctx);
        if (ev) cudaEventRecord(ev->first, ctx->stream);
        EFE_TRY(efe_tc_cells(ctx, Xb, ldb, N, Ycells, ldy, ctx->d_err));
        if (ev) cudaEventRecord(ev->second, ctx->stream);
    }
    const float *Ye = Y + nn * N;
    if (cpl) {
        dim3 gr(s.nch, ctx->natoms);
        k_support_reduce<__nv_bfloat16><<<gr, 128, 0, ctx->stream>>>(
            ctx->d_sup_off, ctx->d_sup_node, ctx->enrich ? ctx->d_Hca : ctx->d_Pc,
            (ctx->enrich && ctx->nonlocal) ? ctx->d_Pc : nullptr, Xb, N, ldb, s.chunk, s.nch, s.part);
        long long n8 = (long long)ctx->natoms * 8 * N;
        k_support_sum<<<nblk(n8, 256), 256, 0, ctx->stream>>>(ctx->natoms, s.nch, N, s.part,
                                                              ctx->enrich ? s.Rh : s.Wc,
                                                              (ctx->enrich && ctx->nonlocal) ? s.Wc : nullptr);
        ctx->launches += 2;
        if (ctx->nonlocal) {
            k_proj_w<float><<<nblk((long long)ctx->n_proj * N, 256), 256, 0, ctx->stream>>>(
                ctx->n_proj, ctx->n_enr, s.Wc, ctx->enrich ? ctx->d_Pa : nullptr, Ye, N, ctx->d_hproj, N, s.W);
            ctx->launches++;
        }
        if (ctx->enrich) {
            k_enr_raw<float><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(
                ctx->n_enr, ctx->n_proj, s.Rh, ctx->d_Haa, ctx->nonlocal ? ctx->d_Pa : nullptr, s.W, Ye, N, N, s.Yraw);
            ctx->launches++;
        }
    }
    k_gather<<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(m, nn, N, Ycells, ldy, cpl ? ctx->d_node_ptr : nullptr,
                                                         ctx->d_node_ent, ctx->d_ent_atom, ctx->d_Hca, ctx->d_Pc, Ye,
                                                         s.W, ctx->enrich ? 1 : 0, ctx->nonlocal ? 1 : 0, HY);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_gather"));
    if (ctx->enrich) {
        dim3 gr(s.nch, ctx->natoms);
        k_support_reduce<float><<<gr, 128, 0, ctx->stream>>>(ctx->d_sup_off, ctx->d_sup_node, ctx->d_C, nullptr, HY,
                                                             N, N, s.chunk, s.nch, s.part);
        long long n8 = (long long)ctx->natoms * 8 * N;
        k_support_sum<<<nblk(n8, 256), 256, 0, ctx->stream>>>(ctx->natoms, s.nch, N, s.part, s.Q, nullptr);
        k_enr_final<float><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(ctx->n_enr, N, s.Yraw, s.Q,
                                                                                           HY + nn * N, N);
        ctx->launches += 3;
    }
    return efe_check_launch(ctx, "hx_bf16");
}

// ===========================================================================
// products used by the drivers
// ===========================================================================
template <typename T>
static efe_status mtilde_inv(efe_ctx *ctx, const T *X, T *Y, int N) {
    const long long nn = ctx->n_nodes;
    k_diag_scale<T><<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(nn, N, ctx->d_minv, X, Y);
    ctx->launches++;
    if (ctx->n_enr) {
        k_enr_mat<T><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(ctx->n_enr, N, ctx->d_Mblk_inv, 1,
                                                                                    X + nn * N, Y + nn * N);
        ctx->launches++;
    }
    return efe_check_launch(ctx, "mtilde_inv");
}

// M~ (the block-diagonal approximation itself) or exact M^E (full M^ee)
static efe_status m_apply(efe_ctx *ctx, const double *X, double *Y, int N, bool exact) {
    const long long nn = ctx->n_nodes;
    k_diag_scale<double><<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(nn, N, ctx->d_mcc, X, Y);
    ctx->launches++;
    if (ctx->n_enr) {
        if (exact)
            k_enr_mat<double><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(
                ctx->n_enr, N, ctx->d_Mee, 0, X + nn * N, Y + nn * N);
        else
            k_enr_mat<double><<<nblk((long long)ctx->n_enr * N, 256), 256, 0, ctx->stream>>>(
                ctx->n_enr, N, ctx->d_Mblk, 1, X + nn * N, Y + nn * N);
        ctx->launches++;
    }
    return efe_check_launch(ctx, "m_apply");
}

efe_status efe_hx(efe_ctx *ctx, const double *X, double *Y, int N, efe_precision prec, double *wsXp) {
    (void)prec;
    return hx_generic<double>(ctx, X, Y, N, ctx->d_He, wsXp);
}
efe_status efe_mx(efe_ctx *ctx, const double *X, double *Y, int N) { return m_apply(ctx, X, Y, N, true); }
efe_status efe_minvx(efe_ctx *ctx, const double *X, double *Y, int N) { return mtilde_inv<double>(ctx, X, Y, N); }

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        return ms;
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// scratch carving from the big workspace
struct Carver {
    char *p;
    size_t left;
    template <typename T>
    T *take(size_t n) {
        size_t bytes = ((n * sizeof(T)) + 255) & ~size_t(255);
        T *r = reinterpret_cast<T *>(p);
        p += bytes;
        left -= bytes;
        return r;
    }
};

template <typename T>
efe_status filter_impl(efe_ctx *ctx, const double *V, const double *HV, const double *lam_dev, int N, int m,
                       const double bounds[3], double *Vout, bool standard = false) {
    const long long rows = ctx->n_rows, nn = ctx->n_nodes;
    const long long n = rows * N;
    const double a0 = bounds[0], a = bounds[1], b = bounds[2];
    if (!(b > a) || !(a0 < a)) {
        ctx->err = "filter bounds must satisfy a0 < a < b";
        return EFE_ERR_ARG;
    }
    std::vector<double> lam(N, 0.0);   // the standard filter passes no Ritz values
    if (lam_dev) {
        EFE_CUDA(ctx, cudaMemcpyAsync(lam.data(), lam_dev, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    std::vector<double> ck, sig;
    cheb_table(m, N, lam.data(), a, b, a0, ck, sig);
    // the standard filter has no forcing term and no V diag(C_m) part
    if (standard) std::fill(ck.begin(), ck.end(), 0.0);
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    size_t need = 256 * 16 + sizeof(double) * (2 * n + (size_t)(m + 1) * N) + sizeof(T) * (5 * n + nn * N);
    EFE_TRY(efe_workspace(ctx, need));
    Carver cv{(char *)ctx->d_ws, ctx->ws_bytes};
    double *G = cv.take<double>(n), *MV = cv.take<double>(n), *dck = cv.take<double>((size_t)(m + 1) * N);
    T *Z0 = cv.take<T>(n), *Z1 = cv.take<T>(n), *Z2 = cv.take<T>(n), *Y = cv.take<T>(n), *HY = cv.take<T>(n);
    T *Xp = cv.take<T>((size_t)nn * N);
    EFE_CUDA(ctx, cudaMemcpyAsync(dck, ck.data(), sizeof(double) * ck.size(), cudaMemcpyHostToDevice, ctx->stream));
    ctx->cell_events_used = 0;
    ctx->cell_launches = 0;
    Timer tm(ctx->stream);
    const long long l0 = ctx->launches;
    T *Zprev = nullptr, *Zcur = Z1, *Znext = Z2, *Zspare = Z0;
    if (standard) {
        EFE_TRY(m_apply(ctx, V, MV, N, false));
        k_std_start<T><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, c, sig[1] / e, HV, MV, G, Z0, Z1);
        ctx->launches++;
        Zprev = Z0;
    } else {
        EFE_TRY(m_apply(ctx, V, MV, N, true));
        k_eig_residual<<<nblk(n, 256), 256, 0, ctx->stream>>>(rows, N, HV, MV, lam_dev, G);
        k_scale_to<T><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, sig[1] / e, G, Z1);
        ctx->launches += 2;
    }
    const T *He = std::is_same<T, double>::value ? (const T *)ctx->d_He : (const T *)ctx->d_He32;
    for (int k = 2; k <= m; ++k) {
        EFE_TRY(mtilde_inv<T>(ctx, Zcur, Y, N));
        EFE_TRY(hx_generic<T>(ctx, Y, HY, N, He, Xp));
        const double ak = 2.0 * sig[k] / e, bk = sig[k - 1] * sig[k];
        k_recurrence<T><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, N, ak, c, bk, HY, Zcur, Zprev, G,
                                                               dck + (size_t)(k - 1) * N, Znext);
        ctx->launches++;
        EFE_TRY(efe_check_launch(ctx, "k_recurrence"));
        T *old_prev = Zprev ? Zprev : Zspare;
        Zprev = Zcur;
        Zcur = Znext;
        Znext = old_prev;
    }
    EFE_TRY(mtilde_inv<T>(ctx, Zcur, Y, N));
    k_vout<T><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, N, Y, V, dck + (size_t)m * N, Vout);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_vout"));
    ctx->stats.ms_filter = tm.stop();
    ctx->stats.ms_cell = cell_events_ms(ctx);
    ctx->stats.launches = ctx->launches - l0;
    ctx->stats.cell_launches = ctx->cell_launches;
    return EFE_OK;
}

}  // namespace

// Residual filter with tcgen05 cell products (bf16 operands, FP32 accumulate).
// The recurrence runs in the variables Y = M~^-1 Z: the FE rows of Y_k are
// exactly the B operand of the next cell products, so they are stored once,
// in bf16, and read by TMA with no separate operand pass; Ghat = (M^cc)^-1 G
// likewise.  The enriched rows keep Z in FP32 (a few hundred rows).  All
// arithmetic is FP32 (FP32 accumulation in the products and the sums); G,
// V_out and the Chebyshev scalars are formed in FP64 as in filter_impl.  Per
// recurrence step: Y_e = (M~^ee)^-1 Z_e, the tensor-core cell products, the
// coupling reductions E Y_c, P_c Y_c over the supports, the enriched rows, and
// the fused gather + recurrence of the FE rows.
static efe_status filter_tensor(efe_ctx *ctx, const double *V, const double *HV, const double *lam_dev, int N,
                                int m, const double bounds[3], double *Vout, bool standard) {
    const MeshDev &mh = ctx->m;
    const long long rows = ctx->n_rows, nn = ctx->n_nodes;
    const int ne_ = ctx->n_enr;
    const double a0 = bounds[0], a = bounds[1], b = bounds[2];
    if (!(b > a) || !(a0 < a)) {
        ctx->err = "filter bounds must satisfy a0 < a < b";
        return EFE_ERR_ARG;
    }
    if (nn > 2147483647LL) {
        ctx->err = "mesh too large for 32-bit node indices";
        return EFE_ERR_ARG;
    }
    if ((long long)mh.nx * mh.ny * mh.nz * mh.ne > 2147483647LL) {
        ctx->err = "mesh too large for 32-bit cell-row indices";
        return EFE_ERR_ARG;
    }
    if (N > 256) {
        ctx->err = "the tensor-core filter takes at most 256 columns per call";
        return EFE_ERR_ARG;
    }
    if (!ctx->he16_valid) EFE_TRY(efe_tc_prepare(ctx));
    std::vector<double> lam(N, 0.0);   // the standard filter passes no Ritz values
    if (lam_dev) {
        EFE_CUDA(ctx, cudaMemcpyAsync(lam.data(), lam_dev, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    std::vector<double> ck, sig;
    cheb_table(m, N, lam.data(), a, b, a0, ck, sig);
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    // the standard filter: no forcing term, no V diag(C_m) part, and the start
    // residual formed with the constant c in place of the Ritz values
    std::vector<double> cvec;
    if (standard) {
        std::fill(ck.begin(), ck.end(), 0.0);
        cvec.assign(N, c);
    }
    // one row stride for every filter buffer: 8 bf16 = 16 B (TMA rows), and a
    // multiple of 4 floats for the FP32 rows
    const int ldb = (N + 7) / 8 * 8;
    std::vector<float> ckf((size_t)(m + 1) * ldb, 0.f);
    for (int k = 0; k <= m; ++k)
        for (int j = 0; j < N; ++j) ckf[(size_t)k * ldb + j] = (float)ck[(size_t)k * N + j];
    const long long ncells = (long long)mh.nx * mh.ny * mh.nz;
    const bool cells16 = ctx->cells_bf16;
    const size_t nb = (size_t)nn * ldb, neb = (size_t)std::max(ne_, 1) * ldb + 8,
                 npb = (size_t)std::max(ctx->n_proj, 1) * ldb + 8;
    const size_t ycells = (size_t)ncells * mh.ne * ldb;
    const bool cpl = (ctx->enrich || ctx->nonlocal) && ctx->natoms > 0;
    // the coupling table read by the cell products: every column chunk they may read
    const int nCB = efe_tc_columns(ctx, N, ldb) / 8;
    const size_t nyw = cpl ? (size_t)(ctx->natoms + 1) * nCB * 64 : 64;
    // E Y_c from the padding rows of the cell products: 4 rows per atom slot
    const bool epad = cpl && ctx->epad && ctx->cx_built;
    const size_t nep = epad ? (size_t)ctx->ca_pairs * 4 * ldb : 64;
    size_t need = 32768 + sizeof(double) * ((size_t)std::max(ne_, 1) * N + (size_t)(m + 2) * N) +
                  sizeof(float) * ckf.size() +
                  2 * 4 * nb + sizeof(float) * (5 * neb + npb + nep) + 2 * (neb + npb + nyw) +
                  (cells16 ? 2 : 4) * ycells;
    const size_t nhe = (size_t)std::max(ne_, 1) * std::max(ne_, 1), npe = (size_t)std::max(ctx->n_proj, 1) * std::max(ne_, 1);
    need += sizeof(float) * (nhe + npe) + 64;
    EFE_TRY(efe_workspace(ctx, need));
    Carver cv{(char *)ctx->d_ws, ctx->ws_bytes};
    double *MV = cv.take<double>((size_t)std::max(ne_, 1) * N), *dck = cv.take<double>((size_t)(m + 1) * N);
    double *dc = cv.take<double>((size_t)N);
    float *fck = cv.take<float>(ckf.size());
    __nv_bfloat16 *Yb[3], *Gb;
    for (auto &y : Yb) y = cv.take<__nv_bfloat16>(nb);
    Gb = cv.take<__nv_bfloat16>(nb);
    float *Ze[3], *Ge;
    for (auto &z : Ze) z = cv.take<float>(neb);
    Ge = cv.take<float>(neb);
    float *Ye = cv.take<float>(neb);
    float *W32 = cv.take<float>(npb);
    __nv_bfloat16 *Ye16 = cv.take<__nv_bfloat16>(neb);
    __nv_bfloat16 *W16 = cv.take<__nv_bfloat16>(npb);
    __nv_bfloat16 *YW = cv.take<__nv_bfloat16>(nyw);
    float *Epart = cv.take<float>(nep);
    void *Ycells = cells16 ? (void *)cv.take<__nv_bfloat16>(ycells) : (void *)cv.take<float>(ycells);
    float *HEee32 = cv.take<float>(nhe), *PE32 = cv.take<float>(npe);   // FP32 copies for the enriched rows
    EFE_CUDA(ctx, cudaMemcpyAsync(dck, ck.data(), sizeof(double) * ck.size(), cudaMemcpyHostToDevice, ctx->stream));
    EFE_CUDA(ctx, cudaMemcpyAsync(fck, ckf.data(), sizeof(float) * ckf.size(), cudaMemcpyHostToDevice, ctx->stream));
    if (standard)
        EFE_CUDA(ctx, cudaMemcpyAsync(dc, cvec.data(), sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
    EFE_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    // padding columns of the small enriched-row buffers are read as zeros
    EFE_CUDA(ctx, cudaMemsetAsync(Ye, 0, sizeof(float) * neb, ctx->stream));
    EFE_CUDA(ctx, cudaMemsetAsync(W32, 0, sizeof(float) * npb, ctx->stream));
    EFE_CUDA(ctx, cudaMemsetAsync(Ye16, 0, 2 * neb, ctx->stream));
    EFE_CUDA(ctx, cudaMemsetAsync(W16, 0, 2 * npb, ctx->stream));
    if (cpl && ctx->enrich) {
        k_d2f<<<nblk((long long)nhe, 256), 256, 0, ctx->stream>>>((long long)ne_ * ne_, ctx->d_HEee, HEee32);
        ctx->launches++;
        if (ctx->nonlocal && ctx->d_PE) {
            k_d2f<<<nblk((long long)npe, 256), 256, 0, ctx->stream>>>((long long)ctx->n_proj * ne_, ctx->d_PE, PE32);
            ctx->launches++;
        }
    }
    HxScratch s{};
    int pnch = 0;
    if (cpl) {
        EFE_TRY(hx_scratch(ctx, N, s));
        if (epad) {
            if (ctx->nonlocal) {
                EFE_TRY(p_support_lists(ctx, kPChunk, &pnch));
                if (pnch > s.nch) {   // the partials are sized for the full support lists
                    ctx->err = "projector support chunks exceed the partial-sum buffer";
                    return EFE_ERR_ARG;
                }
            }
        } else {
            EFE_TRY(chunk_order(ctx, s.chunk, s.nch));
        }
    }
    const unsigned rb_all = (unsigned)((rows + 7) / 8);
    const int nruns_x = (mh.Gx + kRun - 1) / kRun;                   // runs of kRun nodes along x
    const unsigned rb_run = (unsigned)(((long long)mh.Gy * mh.Gz * nruns_x + 7) / 8);   // 8 warps per block
    ctx->cell_events_used = 0;
    ctx->rec_events_used = 0;
    ctx->cell_launches = 0;
    Timer tm(ctx->stream);
    const long long l0 = ctx->launches;
    // M V on the enriched rows only (exact M^ee for the residual, its atom blocks
    // for the standard filter); the FE rows' M^cc V is formed inside the start
    if (ne_) {
        k_enr_mat<double><<<nblk((long long)ne_ * N, 256), 256, 0, ctx->stream>>>(
            ne_, N, standard ? ctx->d_Mblk : ctx->d_Mee, standard ? 1 : 0, V + nn * N, MV);
        ctx->launches++;
    }
    k_filter_start_b<<<rb_all, 256, 0, ctx->stream>>>(nn, rows, N, ldb, HV, V, MV, standard ? dc : lam_dev,
                                                      ctx->d_mcc, ctx->d_minv, sig[1] / e, Gb, Yb[1],
                                                      standard ? Yb[0] : nullptr, Ge, Ze[1],
                                                      standard ? Ze[0] : nullptr);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_filter_start_b"));
    int iprev = standard ? 0 : -1, icur = 1, inext = 2;
    for (int k = 2; k <= m; ++k) {
        const float ak = (float)(2.0 * sig[k] / e), bk = (float)(sig[k - 1] * sig[k]), cf = (float)c;
        const __nv_bfloat16 *Ycur = Yb[icur], *Yprev = iprev >= 0 ? Yb[iprev] : nullptr;
        const float *Zcur = Ze[icur], *Zprev = iprev >= 0 ? Ze[iprev] : nullptr;
        if (ne_) {
            k_enr_minv_f<<<nblk((long long)ne_ * N, 256), 256, 0, ctx->stream>>>(ne_, N, ldb, ctx->d_Mblk_inv, Zcur,
                                                                                Ye, ldb, Ye16);
            ctx->launches++;
        }
        if (cpl) {
            if (epad) {
                // P_c Y_c over the projector entries (W is needed by these cell products);
                // E Y_c comes out of their padding rows
                if (ctx->nonlocal) {
                    k_psup_reduce<<<(unsigned)(pnch * std::max(ctx->natoms, 1)), 256, 0, ctx->stream>>>(
                        ctx->d_psup_off, ctx->d_psup_node, reinterpret_cast<const float4 *>(ctx->d_psup_coef), Ycur,
                        N, ldb, pnch, ctx->d_pchunk_order, s.part);
                    const long long n4 = (long long)ctx->natoms * 4 * N;
                    k_support_sum<<<nblk(n4, 256), 256, 0, ctx->stream>>>(ctx->natoms, pnch, N, s.part, s.Wc,
                                                                          nullptr, 4);
                    ctx->launches += 2;
                }
            } else {
                // E Y_c and P_c Y_c over the supports, from the bf16 rows of Y_c
                k_support_reduce3<__nv_bfloat16><<<(unsigned)(s.nch * std::max(ctx->natoms, 1)), 256, 0,
                                                   ctx->stream>>>(
                    ctx->d_sup_off, ctx->d_sup_node, ctx->enrich ? ctx->d_E32 : ctx->d_Pc32,
                    (ctx->enrich && ctx->nonlocal) ? ctx->d_Pc32 : nullptr, Ycur, nullptr, N, ldb, s.chunk, s.nch,
                    ctx->d_chunk_order, s.part);
                const long long n8 = (long long)ctx->natoms * 8 * N;
                k_support_sum<<<nblk(n8, 256), 256, 0, ctx->stream>>>(ctx->natoms, s.nch, N, s.part,
                                                                      ctx->enrich ? s.Rh : s.Wc,
                                                                      (ctx->enrich && ctx->nonlocal) ? s.Wc : nullptr);
                ctx->launches += 2;
            }
            // W = D (P_c Y_c + P^E Y_e)
            if (ctx->nonlocal) {
                k_proj_w_sp<float><<<nblk((long long)ctx->n_proj * N, 256), 256, 0, ctx->stream>>>(
                    ctx->n_proj, ne_, s.Wc, ctx->enrich ? ctx->d_PE : nullptr, Ye, ldb, ctx->d_hproj, N,
                    ctx->d_enbr_ptr, ctx->d_enbr, s.W);
                k_to_float_strided<<<nblk((long long)ctx->n_proj * N, 256), 256, 0, ctx->stream>>>(
                    ctx->n_proj, N, s.W, W32, ldb, W16);
                ctx->launches += 2;
            }
            // the FE rows' coupling E^T Y_e + P_c^T W enters the cell products
            k_pack_yw<<<nblk((long long)(ctx->natoms + 1) * nCB * 64, 256), 256, 0, ctx->stream>>>(
                ctx->natoms, nCB, N, ldb, ctx->enrich ? Ye16 : nullptr, ctx->nonlocal ? W16 : nullptr, YW);
            ctx->launches++;
            EFE_TRY(efe_check_launch(ctx, "coupling"));
        }
        {
            auto *ev = cell_event_pair(ctx);
            if (ev) cudaEventRecord(ev->first, ctx->stream);
            EFE_TRY(efe_tc_cells(ctx, Ycur, ldb, N, Ycells, ldb, ctx->d_err, cells16 ? 1 : 0, cpl ? YW : nullptr,
                                 nCB, epad ? Epart : nullptr));
            if (ev) cudaEventRecord(ev->second, ctx->stream);
        }
        if (cpl && ctx->enrich) {
            // enriched rows: E Y_c + H^E_ee Y_e + P^E^T W
            if (epad) {
                k_epart_sum<<<dim3((unsigned)((N + 31) / 32), 4, (unsigned)ctx->natoms), 256, 0, ctx->stream>>>(
                    N, ldb, ctx->d_atom_pair_off, ctx->d_atom_pairs, Epart, s.Rh);
                ctx->launches++;
            }
            k_enr_raw_f<<<nblk((long long)ne_ * N, 256), 256, 0, ctx->stream>>>(
                ne_, s.Rh, HEee32, (ctx->nonlocal && ctx->d_PE) ? PE32 : nullptr, W32, ldb, Ye, ldb, N,
                ctx->d_enbr_ptr, ctx->d_enbr, s.Yraw);
            ctx->launches++;
            EFE_TRY(efe_check_launch(ctx, "enriched rows"));
        }
        auto *rev = rec_event_pair(ctx);
        if (rev) cudaEventRecord(rev->first, ctx->stream);
        if (cells16)
            k_gather_rec_c<<<rb_run, 256, 0, ctx->stream>>>(mh, nruns_x, ldb, (const __nv_bfloat16 *)Ycells,
                                                            ctx->d_minv, Ycur, Yprev, Gb, fck + (size_t)(k - 1) * ldb,
                                                            ak, cf, bk, Yb[inext]);
        else
            k_gather_rec_b<float><<<rb_run, 256, 0, ctx->stream>>>(
                mh, nruns_x, ldb, (const float *)Ycells, ctx->d_minv, Ycur, Yprev, Gb, fck + (size_t)(k - 1) * ldb,
                ak, cf, bk, Yb[inext]);
        if (rev) cudaEventRecord(rev->second, ctx->stream);
        ctx->launches++;
        EFE_TRY(efe_check_launch(ctx, "node recurrence"));
        if (ne_) {
            k_enr_rec_v<<<nblk((long long)ne_ * ldb, 256), 256, 0, ctx->stream>>>(
                ne_, N, ldb, s.Yraw, nullptr, Zcur, Zprev, Ge, fck + (size_t)(k - 1) * ldb, ak, cf, bk, Ze[inext]);
            ctx->launches++;
        }
        // rotate: Y_{k-1} becomes Y_{k-2}; the old Y_{k-2} (or the unused third buffer) takes Y_{k+1}
        const int old_prev = iprev >= 0 ? iprev : 3 - icur - inext;
        iprev = icur;
        icur = inext;
        inext = old_prev;
    }
    // V_out = M~^-1 Z_m + V diag(C_m(lam))
    if (ne_) {
        k_enr_minv_f<<<nblk((long long)ne_ * N, 256), 256, 0, ctx->stream>>>(ne_, N, ldb, ctx->d_Mblk_inv, Ze[icur],
                                                                            Ye, ldb);
        ctx->launches++;
    }
    k_vout_b<<<rb_all, 256, 0, ctx->stream>>>(nn, rows, N, ldb, Yb[icur], Ye, V, dck + (size_t)m * N, Vout);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "filter_tensor"));
    ctx->stats.ms_filter = tm.stop();
    ctx->stats.ms_cell = cell_events_ms(ctx);
    ctx->stats.rec_launches = (long long)ctx->rec_events_used;
    ctx->stats.ms_rec = rec_events_ms(ctx);
    ctx->stats.launches = ctx->launches - l0;
    ctx->stats.cell_launches = ctx->cell_launches;
    int flag = 0;
    EFE_CUDA(ctx, cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        ctx->err = "tensor-core cell product: a bounded wait gave up (role " + std::to_string(flag) + ")";
        return EFE_ERR_TIMEOUT;
    }
    return EFE_OK;
}

// columns c0 .. c0 + nc - 1 of a rows x N block <-> a rows x nc block
__global__ void k_cols_gather(long long rows, int N, int c0, int nc, const double *X, double *Xb) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * nc) return;
    const long long r = idx / nc;
    Xb[idx] = X[r * N + c0 + (int)(idx - r * nc)];
}
__global__ void k_cols_scatter(long long rows, int N, int c0, int nc, const double *Xb, double *X) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= rows * nc) return;
    const long long r = idx / nc;
    X[r * N + c0 + (int)(idx - r * nc)] = Xb[idx];
}

// The mixed filter takes at most 256 columns per pass (one or two column
// chunks of the cell products); wider blocks go through it in balanced column
// blocks (each column's filter is independent of the others): gathered into
// a contiguous block, filtered, scattered back.
constexpr int kTcMaxCols = 256;
static efe_status filter_tensor_blocked(efe_ctx *ctx, const double *V, const double *HV, const double *lam, int N,
                                        int m, const double bounds[3], double *Vout, bool standard) {
    if (N <= kTcMaxCols) return filter_tensor(ctx, V, HV, lam, N, m, bounds, Vout, standard);
    const long long rows = ctx->n_rows;
    const int nblk_c = (N + kTcMaxCols - 1) / kTcMaxCols, nb0 = (N + nblk_c - 1) / nblk_c;
    double *buf = nullptr;
    EFE_TRY(efe_alloc(ctx, (void **)&buf, sizeof(double) * (size_t)rows * nb0 * 3));
    double *Vb = buf, *HVb = buf + (size_t)rows * nb0, *Ob = buf + 2 * (size_t)rows * nb0;
    efe_status st = EFE_OK;
    double ms = 0.0, ms_cell = 0.0, ms_rec = 0.0;
    long long launches = 0, cell_launches = 0, rec_launches = 0;
    for (int c0 = 0; c0 < N && st == EFE_OK; c0 += nb0) {
        const int nc = std::min(nb0, N - c0);
        const unsigned g = (unsigned)nblk(rows * nc, 256);
        k_cols_gather<<<g, 256, 0, ctx->stream>>>(rows, N, c0, nc, V, Vb);
        k_cols_gather<<<g, 256, 0, ctx->stream>>>(rows, N, c0, nc, HV, HVb);
        ctx->launches += 2;
        st = filter_tensor(ctx, Vb, HVb, lam ? lam + c0 : nullptr, nc, m, bounds, Ob, standard);
        if (st != EFE_OK) break;
        ms += ctx->stats.ms_filter;
        ms_cell += ctx->stats.ms_cell;
        ms_rec += ctx->stats.ms_rec;
        launches += ctx->stats.launches;
        cell_launches += ctx->stats.cell_launches;
        rec_launches += ctx->stats.rec_launches;
        k_cols_scatter<<<g, 256, 0, ctx->stream>>>(rows, N, c0, nc, Ob, Vout);
        ctx->launches++;
        st = efe_check_launch(ctx, "column blocks");
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(buf);
    if (st == EFE_OK) {
        ctx->stats.ms_filter = ms;
        ctx->stats.ms_cell = ms_cell;
        ctx->stats.ms_rec = ms_rec;
        ctx->stats.launches = launches + 3LL * nblk_c;
        ctx->stats.cell_launches = cell_launches;
        ctx->stats.rec_launches = rec_launches;
    }
    return st;
}

efe_status efe_filter_dispatch(efe_ctx *ctx, const double *V, const double *HV, const double *lam, int N, int m,
                               const double bounds[3], efe_precision prec, double *Vout, bool standard = false) {
    if (prec == EFE_FP64) return filter_impl<double>(ctx, V, HV, lam, N, m, bounds, Vout, standard);
    if (prec == EFE_FP32) return filter_impl<float>(ctx, V, HV, lam, N, m, bounds, Vout, standard);
    if (prec == EFE_BF16) return filter_tensor_blocked(ctx, V, HV, lam, N, m, bounds, Vout, standard);
    ctx->err = "unknown precision";
    return EFE_ERR_ARG;
}

// Rayleigh-Ritz (Eq. projectedKSEig), FP64.
efe_status efe_rr_impl(efe_ctx *ctx, double *X, double *HX, int N, double *eig, double *resid) {
    const long long rows = ctx->n_rows, nn = ctx->n_nodes;
    const long long n = rows * N;
    size_t need = 256 * 8 + sizeof(double) * (2 * n + nn * N);
    EFE_TRY(efe_workspace(ctx, need));
    Carver cv{(char *)ctx->d_ws, ctx->ws_bytes};
    double *MX = cv.take<double>(n), *T1 = cv.take<double>(n), *Xp = cv.take<double>((size_t)nn * N);
    Timer tm(ctx->stream);
    k_zero_boundary<<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(ctx->m, nn, N, X);
    ctx->launches++;
    EFE_TRY(hx_generic<double>(ctx, X, HX, N, ctx->d_He, Xp));
    EFE_TRY(m_apply(ctx, X, MX, N, true));
    const long long chunk = 4096;
    const int nch = (int)((rows + chunk - 1) / chunk);
    const size_t N2 = (size_t)N * N;
    EFE_TRY(efe_partials(ctx, (size_t)nch * N2 + 6 * N2 + 4 * N + (size_t)nch * N));
    double *part = ctx->d_part, *S0 = part + (size_t)nch * N2, *H0 = S0 + N2, *Ss = H0 + N2, *Hs = Ss + N2,
           *Qr = Hs + N2, *d = Qr + N2, *W = d + N, *rs = W + N, *rpart = rs + N + N2;
    dim3 g(nch, nblk(N, 32), nblk(N, 32));
    k_gram_partial<<<g, 256, 0, ctx->stream>>>(rows, N, X, MX, chunk, part);
    k_gram_sum<<<nblk(N2, 256), 256, 0, ctx->stream>>>(N, nch, part, S0);
    k_gram_partial<<<g, 256, 0, ctx->stream>>>(rows, N, X, HX, chunk, part);
    k_gram_sum<<<nblk(N2, 256), 256, 0, ctx->stream>>>(N, nch, part, H0);
    ctx->launches += 4;
    EFE_TRY(efe_check_launch(ctx, "gram"));
    k_rr_scale<<<nblk(N2, 256), 256, 0, ctx->stream>>>(N, S0, H0, Ss, Hs, d);
    ctx->launches++;
    EFE_TRY(efe_check_launch(ctx, "k_rr_scale"));
    if (cusolverDnSetStream(ctx->solver, ctx->stream) != CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnSetStream failed";
        return EFE_ERR_CUDA;
    }
    int lwork = 0;
    if (cusolverDnDsygvd_bufferSize(ctx->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                    CUBLAS_FILL_MODE_UPPER, N, Hs, N, Ss, N, W, &lwork) != CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnDsygvd_bufferSize failed";
        return EFE_ERR_CUDA;
    }
    if ((size_t)lwork * 8 > ctx->solver_ws_bytes) {
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->d_solver_ws) cudaFree(ctx->d_solver_ws);
        ctx->d_solver_ws = nullptr;
        ctx->solver_ws_bytes = 0;
        EFE_TRY(efe_alloc(ctx, &ctx->d_solver_ws, (size_t)lwork * 8));
        ctx->solver_ws_bytes = (size_t)lwork * 8;
    }
    if (cusolverDnDsygvd(ctx->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, N, Hs,
                         N, Ss, N, W, (double *)ctx->d_solver_ws, lwork, ctx->d_info) != CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnDsygvd failed";
        return EFE_ERR_CUDA;
    }
    int info = 0;
    EFE_CUDA(ctx, cudaMemcpyAsync(&info, ctx->d_info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (info != 0) {
        ctx->err = "Rayleigh-Ritz: generalized eigensolve failed (sygvd info " + std::to_string(info) +
                   (info > N ? ": X^T M X is not positive definite)" : ": eigenvalues did not converge)");
        return EFE_ERR_NOT_SPD;
    }
    k_rr_unscale<<<nblk(N2, 256), 256, 0, ctx->stream>>>(N, Hs, d, Qr);
    const size_t shm = sizeof(double) * 16 * N;
    cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    const unsigned rb = (unsigned)((rows + 15) / 16);
    k_rotate<<<rb, 256, shm, ctx->stream>>>(rows, N, X, Qr, T1);
    EFE_CUDA(ctx, cudaMemcpyAsync(X, T1, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    k_rotate<<<rb, 256, shm, ctx->stream>>>(rows, N, HX, Qr, T1);
    EFE_CUDA(ctx, cudaMemcpyAsync(HX, T1, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    k_rotate<<<rb, 256, shm, ctx->stream>>>(rows, N, MX, Qr, T1);
    EFE_CUDA(ctx, cudaMemcpyAsync(MX, T1, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    k_resid_partial<<<nch, 128, 0, ctx->stream>>>(rows, N, HX, MX, W, chunk, rpart);
    k_colsum<<<nblk(N, 128), 128, 0, ctx->stream>>>(N, nch, rpart, rs);
    ctx->launches += 6;
    EFE_TRY(efe_check_launch(ctx, "rr rotate"));
    std::vector<double> r2(N);
    EFE_CUDA(ctx, cudaMemcpyAsync(eig, W, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    EFE_CUDA(ctx, cudaMemcpyAsync(r2.data(), rs, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (resid)
        for (int j = 0; j < N; ++j) resid[j] = std::sqrt(std::max(r2[j], 0.0));
    ctx->stats.ms_rr = tm.stop();
    return EFE_OK;
}

// k-step Lanczos for M~^-1 H in the M~ inner product.
static efe_status lanczos_impl(efe_ctx *ctx, const double *u0, int k, double out[3]) {
    const long long rows = ctx->n_rows, nn = ctx->n_nodes;
    size_t need = 256 * 8 + sizeof(double) * (5 * rows + nn);
    EFE_TRY(efe_workspace(ctx, need));
    Carver cv{(char *)ctx->d_ws, ctx->ws_bytes};
    double *q = cv.take<double>(rows), *qp = cv.take<double>(rows), *w = cv.take<double>(rows),
           *r = cv.take<double>(rows), *t = cv.take<double>(rows), *Xp = cv.take<double>(nn);
    const int nb = 256;
    EFE_TRY(efe_partials(ctx, nb));
    Timer tm(ctx->stream);
    std::vector<double> hp(nb);
    auto dot = [&](const double *a, const double *b, double &res) -> efe_status {
        k_dot_partial<<<nb, 256, 0, ctx->stream>>>(rows, a, b, ctx->d_part);
        ctx->launches++;
        EFE_CUDA(ctx, cudaMemcpyAsync(hp.data(), ctx->d_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        res = 0.0;
        for (int i = 0; i < nb; ++i) res += hp[i];
        return EFE_OK;
    };
    EFE_TRY(m_apply(ctx, u0, t, 1, false));
    double nrm2;
    EFE_TRY(dot(u0, t, nrm2));
    if (!(nrm2 > 0.0)) {
        ctx->err = "Lanczos start vector has zero norm";
        return EFE_ERR_ARG;
    }
    k_axpby3<<<nblk(rows, 256), 256, 0, ctx->stream>>>(rows, 1.0 / std::sqrt(nrm2), u0, 0.0, u0, 0.0, nullptr, q);
    EFE_CUDA(ctx, cudaMemsetAsync(qp, 0, sizeof(double) * rows, ctx->stream));
    std::vector<double> al, be;
    double beta = 0.0;
    for (int j = 0; j < k; ++j) {
        EFE_TRY(hx_generic<double>(ctx, q, w, 1, ctx->d_He, Xp));
        double alpha;
        EFE_TRY(dot(q, w, alpha));
        EFE_TRY(mtilde_inv<double>(ctx, w, r, 1));
        k_axpby3<<<nblk(rows, 256), 256, 0, ctx->stream>>>(rows, 1.0, r, -alpha, q, -beta, qp, r);
        EFE_TRY(m_apply(ctx, r, t, 1, false));
        double b2;
        EFE_TRY(dot(r, t, b2));
        beta = std::sqrt(std::max(b2, 0.0));
        al.push_back(alpha);
        be.push_back(beta);
        if (beta == 0.0) break;
        std::swap(qp, q);
        k_axpby3<<<nblk(rows, 256), 256, 0, ctx->stream>>>(rows, 1.0 / beta, r, 0.0, r, 0.0, nullptr, q);
        ctx->launches += 2;
    }
    const int kk = (int)al.size();
    std::vector<double> Tm(kk * kk, 0.0), wv, Vv;
    for (int i = 0; i < kk; ++i) {
        Tm[i * kk + i] = al[i];
        if (i + 1 < kk) Tm[i * kk + i + 1] = Tm[(i + 1) * kk + i] = be[i];
    }
    jacobi_eig(kk, Tm, wv, Vv);
    int imin = 0, imax = 0;
    for (int i = 1; i < kk; ++i) {
        if (wv[i] < wv[imin]) imin = i;
        if (wv[i] > wv[imax]) imax = i;
    }
    out[0] = wv[imin];
    out[1] = wv[imax];
    out[2] = wv[imax] + std::fabs(be[kk - 1] * Vv[(kk - 1) * kk + imax]);
    ctx->stats.ms_lanczos = tm.stop();
    return EFE_OK;
}

// ---- helpers used by the SCF translation unit -------------------------------
efe_status efe_cells_shared(efe_ctx *ctx, const double *K, const double *X, double *Y, int N) {
    EFE_CUDA(ctx, cudaMemsetAsync(Y, 0, sizeof(double) * ctx->n_nodes * N, ctx->stream));
    // not bracketed by the cell-product timing events, which the filter's statistics report
    return launch_cells<double>(ctx, K, 0, X, Y, N, N, false);
}
efe_status efe_xprime_fp64(efe_ctx *ctx, const double *X, double *Xp, int N) {
    const long long nn = ctx->n_nodes;
    k_xprime<double><<<nblk(nn * N, 256), 256, 0, ctx->stream>>>(ctx->m, nn, X, Xp, N, N, ctx->d_node_ptr,
                                                                 ctx->d_node_ent, ctx->d_ent_atom, ctx->d_C,
                                                                 ctx->enrich ? 1 : 0);
    ctx->launches++;
    return efe_check_launch(ctx, "k_xprime");
}
void efe_sym_eig(int n, const std::vector<double> &A, std::vector<double> &w, std::vector<double> &V) {
    jacobi_eig(n, A, w, V);
}

// ===========================================================================
// C ABI
// ===========================================================================
static thread_local std::string g_setup_err;

#define EFE_CHECK_CTX(ctx)                                  \
    do {                                                    \
        if (!(ctx)) return EFE_ERR_ARG;                     \
    } while (0)
#define EFE_ARG(ctx, cond, msg)                             \
    do {                                                    \
        if (!(cond)) {                                      \
            (ctx)->err = (msg);                             \
            return EFE_ERR_ARG;                             \
        }                                                   \
    } while (0)

extern "C" {

const char *efe_last_error(const efe_ctx *ctx) { return ctx ? ctx->err.c_str() : g_setup_err.c_str(); }

void efe_destroy(efe_ctx *ctx) {
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    efe_scf_free(ctx);
    void *ptrs[] = {ctx->d_chunk_order, ctx->d_nm_atom, ctx->d_nm_E32, ctx->d_nm_P32, ctx->d_E, ctx->d_PE, ctx->d_HEee, ctx->d_hostio, ctx->d_B1, ctx->d_D1, ctx->d_wq, ctx->d_Khat, ctx->d_mcc, ctx->d_minv, ctx->d_He, ctx->d_He32,
                    ctx->d_He16, ctx->d_atoms, ctx->d_hproj, ctx->d_sup_off, ctx->d_sup_node, ctx->d_C, ctx->d_B,
                    ctx->d_Kca, ctx->d_Hca, ctx->d_Pc, ctx->d_E32, ctx->d_Pc32, ctx->d_node_ptr,
                    ctx->d_node_ent, ctx->d_ent_atom,
                    ctx->d_pairs, ctx->d_pair_pos, ctx->d_cell_atom_ptr, ctx->d_cell_atoms, ctx->d_Aee, ctx->d_Kaa,
                    ctx->d_Haa, ctx->d_Mee, ctx->d_Pa, ctx->d_Mblk_inv, ctx->d_Mblk, ctx->d_ws, ctx->d_part,
                    ctx->d_info, ctx->d_err, ctx->d_solver_ws, ctx->d_cx_off, ctx->d_cx_atoms, ctx->d_Ax,
                    ctx->d_atom_pair_off, ctx->d_atom_pairs, ctx->d_psup_off, ctx->d_psup_node,
                    ctx->d_psup_coef, ctx->d_pchunk_order, ctx->d_enbr_ptr, ctx->d_enbr};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    for (auto *ev : {&ctx->cell_events, &ctx->rec_events})
        for (auto &e : *ev) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
    if (ctx->solver) cusolverDnDestroy(ctx->solver);
    delete ctx;
}

efe_status efe_setup(const efe_mesh *mesh, const efe_atoms *atoms, const efe_enrichment *enrich,
                     const efe_psp *psp, void *stream, efe_ctx **out) {
    g_setup_err.clear();
    if (!out || !mesh || !atoms) {
        g_setup_err = "efe_setup: null argument";
        return EFE_ERR_ARG;
    }
    *out = nullptr;
    auto fail = [&](const char *msg) {
        g_setup_err = msg;
        return EFE_ERR_ARG;
    };
    if (!(mesh->h > 0.0)) return fail("mesh h must be > 0");
    if (mesh->degree < 1 || mesh->degree > EFE_MAXP) return fail("degree must be in [1, 8]");
    for (int d = 0; d < 3; ++d)
        if (mesh->ncell[d] < 1) return fail("ncell must be >= 1");
    const int nq = mesh->nquad > 0 ? mesh->nquad : mesh->degree + 2;
    if (nq > EFE_MAXNQ || nq < mesh->degree + 1) return fail("nquad must be in [p+1, 12]");
    if (atoms->natoms < 0 || (atoms->natoms > 0 && (!atoms->xyz || !atoms->zval))) return fail("bad atoms");
    const bool en = enrich && enrich->enabled;
    const bool nl = psp && psp->enabled;
    if (en && !(enrich->alpha > 0.0 && enrich->r_end > 0.0 && enrich->t > 0.0)) return fail("bad enrichment");
    if (nl && (!(psp->rc > 0.0) || !(psp->r_trunc > 0.0) || (atoms->natoms > 0 && !psp->h)))
        return fail("bad pseudopotential");
    efe_ctx *ctx = new efe_ctx();
    ctx->stream = (cudaStream_t)stream;
    MeshDev &m = ctx->m;
    m.nx = mesh->ncell[0];
    m.ny = mesh->ncell[1];
    m.nz = mesh->ncell[2];
    m.p = mesh->degree;
    m.np1 = m.p + 1;
    m.ne = m.np1 * m.np1 * m.np1;
    m.nq = nq;
    m.nq3 = nq * nq * nq;
    m.h = mesh->h;
    m.Gx = m.nx * m.p + 1;
    m.Gy = m.ny * m.p + 1;
    m.Gz = m.nz * m.p + 1;
    ctx->natoms = atoms->natoms;
    ctx->enrich = en && atoms->natoms > 0;
    ctx->nonlocal = nl && atoms->natoms > 0;
    ctx->n_enr = ctx->enrich ? 4 * ctx->natoms : 0;
    ctx->n_proj = ctx->nonlocal ? 4 * ctx->natoms : 0;
    ctx->n_nodes = (long long)m.Gx * m.Gy * m.Gz;
    ctx->n_rows = ctx->n_nodes + ctx->n_enr;
    ctx->n_fe_dof = (long long)(m.Gx - 2) * (m.Gy - 2) * (m.Gz - 2);
    ctx->n_quad = (long long)m.nx * m.ny * m.nz * m.nq3;
    if (ctx->enrich) {
        ctx->alpha = enrich->alpha;
        ctx->t = enrich->t;
        ctx->r0 = enrich->r_end * enrich->t / (1.0 + enrich->t);
    }
    if (ctx->nonlocal) {
        ctx->rc = psp->rc;
        ctx->rtrunc = psp->r_trunc;
    }
    if (psp) ctx->rloc = psp->rloc > 0 ? psp->rloc : 0.8;
    ctx->xyz.assign(atoms->xyz, atoms->xyz + 3 * atoms->natoms);
    ctx->zval.assign(atoms->zval, atoms->zval + atoms->natoms);
    const double L[3] = {m.nx * m.h, m.ny * m.h, m.nz * m.h};
    for (int I = 0; I < ctx->natoms; ++I)
        for (int d = 0; d < 3; ++d) {
            double x = ctx->xyz[3 * I + d];
            if (x < 0.0 || x > L[d]) { delete ctx; return fail("atom outside the box"); }
            if (ctx->enrich && (x - enrich->r_end < -1e-12 || x + enrich->r_end > L[d] + 1e-12)) {
                delete ctx;
                return fail("enrichment support leaves the box (Dirichlet boundary)");
            }
        }
    auto bail = [&](efe_status st) {
        g_setup_err = ctx->err;
        efe_destroy(ctx);
        return st;
    };
    efe_status st;
    if (cudaGetDevice(&ctx->device) != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        ctx->err = "invalid CUDA stream or no device";
        return bail(EFE_ERR_CUDA);
    }
    if (cusolverDnCreate(&ctx->solver) != CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnCreate failed";
        return bail(EFE_ERR_CUDA);
    }
    if ((st = efe_alloc(ctx, (void **)&ctx->d_info, sizeof(int))) != EFE_OK) return bail(st);
    if ((st = efe_alloc(ctx, (void **)&ctx->d_err, sizeof(int))) != EFE_OK) return bail(st);
    if (cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) return bail(EFE_ERR_CUDA);
    if ((st = efe_alloc(ctx, (void **)&ctx->d_atoms, sizeof(double) * 3 * std::max(1, ctx->natoms))) != EFE_OK)
        return bail(st);
    if (ctx->natoms && cudaMemcpy(ctx->d_atoms, ctx->xyz.data(), sizeof(double) * 3 * ctx->natoms,
                                  cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(EFE_ERR_CUDA);
    if (ctx->nonlocal) {
        ctx->hproj.assign(psp->h, psp->h + 2 * ctx->natoms);
        std::vector<double> D(ctx->n_proj);
        for (int I = 0; I < ctx->natoms; ++I) {
            D[4 * I] = ctx->hproj[2 * I];
            for (int mm = 1; mm < 4; ++mm) D[4 * I + mm] = ctx->hproj[2 * I + 1];
        }
        if ((st = efe_alloc(ctx, (void **)&ctx->d_hproj, sizeof(double) * ctx->n_proj)) != EFE_OK) return bail(st);
        if (cudaMemcpy(ctx->d_hproj, D.data(), sizeof(double) * ctx->n_proj, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(EFE_ERR_CUDA);
    }
    if ((st = efe_build_tables(ctx)) != EFE_OK) return bail(st);
    if ((st = efe_static_integrals(ctx)) != EFE_OK) return bail(st);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        ctx->err = std::string("setup: ") + cudaGetErrorString(cudaGetLastError());
        return bail(EFE_ERR_CUDA);
    }
    *out = ctx;
    return EFE_OK;
}

efe_status efe_get_dims(const efe_ctx *ctx, efe_dims *d) {
    if (!ctx || !d) return EFE_ERR_ARG;
    d->n_nodes = ctx->n_nodes;
    d->n_fe_dof = ctx->n_fe_dof;
    d->n_rows = ctx->n_rows;
    d->n_quad = ctx->n_quad;
    d->n_enr = ctx->n_enr;
    d->n_proj = ctx->n_proj;
    d->n_cells = ctx->m.nx * ctx->m.ny * ctx->m.nz;
    d->ne = ctx->m.ne;
    d->nq = ctx->m.nq;
    d->grid[0] = ctx->m.Gx;
    d->grid[1] = ctx->m.Gy;
    d->grid[2] = ctx->m.Gz;
    d->n_support_nodes = ctx->n_support_nodes;
    return EFE_OK;
}

efe_status efe_get_stats(const efe_ctx *ctx, efe_stats *s) {
    if (!ctx || !s) return EFE_ERR_ARG;
    *s = ctx->stats;
    return EFE_OK;
}

efe_status efe_set_cell_storage(efe_ctx *ctx, efe_precision prec) {
    EFE_CHECK_CTX(ctx);
    if (prec != EFE_BF16 && prec != EFE_FP32) {
        ctx->err = "efe_set_cell_storage: EFE_BF16 or EFE_FP32";
        return EFE_ERR_ARG;
    }
    ctx->cells_bf16 = prec == EFE_BF16;
    return EFE_OK;
}

efe_status efe_set_potential(efe_ctx *ctx, const double *veff_q) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, veff_q, "veff_q is null");
    EFE_TRY(efe_potential_assembly(ctx, veff_q));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

efe_status efe_apply_h(efe_ctx *ctx, const double *X, double *Y, int N, efe_precision prec) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, X && Y && X != Y && N > 0, "efe_apply_h: bad arguments");
    if (!ctx->have_potential) {
        ctx->err = "efe_apply_h: no potential set";
        return EFE_ERR_STATE;
    }
    const long long n = ctx->n_rows * N;
    if (prec == EFE_FP64) {
        EFE_TRY(efe_workspace(ctx, sizeof(double) * ctx->n_nodes * N + 256));
        return hx_generic<double>(ctx, X, Y, N, ctx->d_He, (double *)ctx->d_ws);
    }
    if (prec == EFE_FP32) {
        EFE_TRY(efe_workspace(ctx, sizeof(float) * (2 * n + ctx->n_nodes * N) + 1024));
        Carver cv{(char *)ctx->d_ws, ctx->ws_bytes};
        float *Xf = cv.take<float>(n), *Yf = cv.take<float>(n), *Xp = cv.take<float>((size_t)ctx->n_nodes * N);
        k_cast<double, float><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, X, Xf);
        EFE_TRY(hx_generic<float>(ctx, Xf, Yf, N, ctx->d_He32, Xp));
        k_cast<float, double><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, Yf, Y);
        return efe_check_launch(ctx, "apply_h fp32");
    }
    if (prec == EFE_BF16) {
        const int ldb = (N + 7) / 8 * 8, ldy = (N + 3) / 4 * 4;
        const long long ncells = (long long)ctx->m.nx * ctx->m.ny * ctx->m.nz;
        EFE_TRY(efe_workspace(ctx, sizeof(float) * 2 * n + 2 * (size_t)ctx->n_nodes * ldb +
                                       4 * (size_t)ncells * ctx->m.ne * ldy + 2048));
        Carver cv{(char *)ctx->d_ws, ctx->ws_bytes};
        float *Xf = cv.take<float>(n), *Yf = cv.take<float>(n);
        __nv_bfloat16 *Xb = cv.take<__nv_bfloat16>((size_t)ctx->n_nodes * ldb);
        float *Yc = cv.take<float>((size_t)ncells * ctx->m.ne * ldy);
        EFE_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
        k_cast<double, float><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, X, Xf);
        EFE_TRY(hx_bf16(ctx, Xf, Yf, N, Xb, Yc));
        k_cast<float, double><<<nblk(n, 256), 256, 0, ctx->stream>>>(n, Yf, Y);
        EFE_TRY(efe_check_launch(ctx, "apply_h bf16"));
        int flag = 0;
        EFE_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (flag) {
            ctx->err = "tensor-core cell product: a bounded wait gave up";
            return EFE_ERR_TIMEOUT;
        }
        return EFE_OK;
    }
    ctx->err = "efe_apply_h: precision not available";
    return EFE_ERR_ARG;
}

efe_status efe_apply_m(efe_ctx *ctx, const double *X, double *Y, int N) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, X && Y && X != Y && N > 0, "efe_apply_m: bad arguments");
    return m_apply(ctx, X, Y, N, true);
}

efe_status efe_apply_minv(efe_ctx *ctx, const double *X, double *Y, int N) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, X && Y && X != Y && N > 0, "efe_apply_minv: bad arguments");
    return mtilde_inv<double>(ctx, X, Y, N);
}

efe_status efe_lanczos(efe_ctx *ctx, const double *u0, int k, double out[3]) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, u0 && out && k >= 1 && k <= 100, "efe_lanczos: bad arguments");
    if (!ctx->have_potential) {
        ctx->err = "efe_lanczos: no potential set";
        return EFE_ERR_STATE;
    }
    return lanczos_impl(ctx, u0, k, out);
}

efe_status efe_filter(efe_ctx *ctx, const double *V, const double *HV, const double *lam, int N, int m,
                      const double bounds[3], efe_precision prec, double *Vout) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, V && HV && lam && bounds && Vout && N > 0 && m >= 1 && Vout != V && Vout != HV,
            "efe_filter: bad arguments");
    if (!ctx->have_potential) {
        ctx->err = "efe_filter: no potential set";
        return EFE_ERR_STATE;
    }
    return efe_filter_dispatch(ctx, V, HV, lam, N, m, bounds, prec, Vout);
}

efe_status efe_filter_standard(efe_ctx *ctx, const double *V, const double *HV, int N, int m,
                               const double bounds[3], efe_precision prec, double *Vout) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, V && HV && bounds && Vout && N > 0 && m >= 1 && Vout != V && Vout != HV,
            "efe_filter_standard: bad arguments");
    if (!ctx->have_potential) {
        ctx->err = "efe_filter_standard: no potential set";
        return EFE_ERR_STATE;
    }
    return efe_filter_dispatch(ctx, V, HV, nullptr, N, m, bounds, prec, Vout, true);
}

efe_status efe_rayleigh_ritz(efe_ctx *ctx, double *X, double *HX, int N, double *eig, double *resid) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, X && HX && eig && N > 0 && X != HX, "efe_rayleigh_ritz: bad arguments");
    if (!ctx->have_potential) {
        ctx->err = "efe_rayleigh_ritz: no potential set";
        return EFE_ERR_STATE;
    }
    return efe_rr_impl(ctx, X, HX, N, eig, resid);
}

efe_status efe_chfsi(efe_ctx *ctx, double *X, double *HX, int N, int m, const double *bounds, const double *u0,
                     int max_pass, double tol, int nconv, efe_precision prec, double *eig, double *resid,
                     int *passes) {
    return efe_chfsi_kind(ctx, X, HX, N, m, bounds, u0, max_pass, tol, nconv, prec, EFE_FILTER_RESIDUAL, eig,
                          resid, passes, nullptr);
}

efe_status efe_chfsi_kind(efe_ctx *ctx, double *X, double *HX, int N, int m, const double *bounds,
                          const double *u0, int max_pass, double tol, int nconv, efe_precision prec, int kind,
                          double *eig, double *resid, int *passes, double *history) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, X && eig && resid && N > 0 && m >= 1 && max_pass >= 0 && (bounds || u0) &&
                     (kind & ~(EFE_FILTER_STANDARD | EFE_FILTER_KEEP_PRECISION)) == 0,
            "efe_chfsi: bad arguments");
    const bool standard = (kind & EFE_FILTER_STANDARD) != 0;
    if (!ctx->have_potential) {
        ctx->err = "efe_chfsi: no potential set";
        return EFE_ERR_STATE;
    }
    if (nconv <= 0 || nconv > N) nconv = N;
    const long long n = ctx->n_rows * N;
    // persistent buffers for HX (if not given), Vout and lam
    double *dHX = HX, *dVout = nullptr, *dlam = nullptr;
    std::vector<void *> owned;
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void *p : owned) cudaFree(p);
    };
    if (!dHX) {
        if (efe_alloc(ctx, (void **)&dHX, sizeof(double) * n) != EFE_OK) return EFE_ERR_OOM;
        owned.push_back(dHX);
    }
    if (efe_alloc(ctx, (void **)&dVout, sizeof(double) * n) != EFE_OK) { cleanup(); return EFE_ERR_OOM; }
    owned.push_back(dVout);
    if (efe_alloc(ctx, (void **)&dlam, sizeof(double) * N) != EFE_OK) { cleanup(); return EFE_ERR_OOM; }
    owned.push_back(dlam);
    double bd[3];
    efe_status st = EFE_OK;
    if (bounds) {
        bd[0] = bounds[0];
        bd[1] = bounds[1];
        bd[2] = bounds[2];
    } else {
        double lz[3];
        if ((st = lanczos_impl(ctx, u0, 10, lz)) != EFE_OK) { cleanup(); return st; }
        bd[0] = lz[0];
        bd[1] = lz[0] + 0.3 * (lz[2] - lz[0]);
        bd[2] = lz[2];
    }
    if ((st = efe_rr_impl(ctx, X, dHX, N, eig, resid)) != EFE_OK) { cleanup(); return st; }
    double ms_filter = 0.0, ms_rr = 0.0;
    int pass = 0;
    bool conv = false;
    // bf16 passes only while they contract the largest wanted residual: the
    // rounding error of a pass scales with the residual, and from a poor
    // subspace of a large problem it can outgrow the filter's damping; after a
    // bf16 pass that does not reduce the residual, the remaining passes are FP32
    efe_precision pp = prec;
    double prev_mx = 0.0;
    for (int j = 0; j < nconv; ++j) prev_mx = std::max(prev_mx, resid[j]);
    while (pass < max_pass) {
        if (cudaMemcpyAsync(dlam, eig, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
            cleanup();
            return EFE_ERR_CUDA;
        }
        if ((st = efe_filter_dispatch(ctx, X, dHX, dlam, N, m, bd, pp, dVout, standard)) != EFE_OK) {
            cleanup();
            return st;
        }
        ms_filter += ctx->stats.ms_filter;
        if ((st = efe_rr_impl(ctx, dVout, dHX, N, eig, resid)) != EFE_OK) { cleanup(); return st; }
        ms_rr += ctx->stats.ms_rr;
        if (cudaMemcpyAsync(X, dVout, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            cleanup();
            return EFE_ERR_CUDA;
        }
        ++pass;
        double mx = 0.0;
        for (int j = 0; j < nconv; ++j) mx = std::max(mx, resid[j]);
        if (history) history[pass - 1] = mx;
        if (pp == EFE_BF16 && !(mx < prev_mx) && !(kind & EFE_FILTER_KEEP_PRECISION)) pp = EFE_FP32;
        prev_mx = mx;
        bd[0] = eig[0];
        bd[1] = eig[N - 1];
        if (mx < tol) { conv = true; break; }
    }
    cleanup();
    ctx->stats.ms_filter = ms_filter;
    ctx->stats.ms_rr = ms_rr;
    ctx->stats.passes = pass;
    if (passes) *passes = pass;
    return (conv || max_pass == 0) ? EFE_OK : EFE_ERR_NO_CONVERGE;
}

efe_status efe_filter_host(efe_ctx *ctx, const double *V, const double *HV, const double *lam, int N, int m,
                           const double bounds[3], efe_precision prec, double *Vout) {
    EFE_CHECK_CTX(ctx);
    EFE_ARG(ctx, V && HV && lam && bounds && Vout && N > 0 && m >= 1, "efe_filter_host: bad arguments");
    const long long n = ctx->n_rows * N;
    // device copies of V, HV, Vout and lam, kept by the context between calls
    const size_t need = sizeof(double) * (3 * (size_t)n + (size_t)N) + 256;
    if (need > ctx->hostio_bytes) {
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->d_hostio) cudaFree(ctx->d_hostio);
        ctx->d_hostio = nullptr;
        ctx->hostio_bytes = 0;
        EFE_TRY(efe_alloc(ctx, &ctx->d_hostio, need));
        ctx->hostio_bytes = need;
    }
    double *dV = static_cast<double *>(ctx->d_hostio), *dHV = dV + n, *dO = dHV + n, *dl = dO + n;
    auto cleanup = [&]() { cudaStreamSynchronize(ctx->stream); };
    efe_status st = EFE_OK;
    if (cudaMemcpyAsync(dV, V, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(dHV, HV, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(dl, lam, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
        ctx->err = "efe_filter_host: host-to-device copy failed";
        cleanup();
        return EFE_ERR_CUDA;
    }
    st = efe_filter(ctx, dV, dHV, dl, N, m, bounds, prec, dO);
    if (st == EFE_OK && cudaMemcpyAsync(Vout, dO, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) {
        ctx->err = "efe_filter_host: device-to-host copy failed";
        st = EFE_ERR_CUDA;
    }
    cleanup();
    return st;
}

}  // extern "C"
