// Learned density warm start: an addition of this library on top of the
// paper's superposition of atomic densities (Sec. II.A, Sec. IV).
//
//   k_descriptors   radial descriptors of every atom (double, stored float)
//   k_mlp           one pass of the 32-128-128-128-8 SiLU network over a tile
//                   of 32 samples per CTA: forward, and for training the
//                   backward pass with the CTA's weight-gradient partials.
//                   The tile's activations stay in shared memory; each
//                   layer's weights are staged there in turn (padded rows,
//                   so that both the forward and the transposed backward
//                   products read them without bank conflicts).
//   k_mlp_reduce    sums the partials in a fixed order; Adam update
//   k_correction    drho at the Gauss points from per-atom coefficients
//   k_fit_rhs, k_fit_gram   normal equations of the least-squares fit
#include "efe_internal.cuh"
#include "efe_funcs.cuh"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

constexpr int ND = EFE_MLP_N_DESC;    // 32 descriptors
constexpr int NH = 128;               // hidden width
constexpr int NO = EFE_MLP_N_OUT;     // 8 coefficients
constexpr int NTRAIN = EFE_MLP_N_TRAIN;
constexpr int NPARAM = EFE_MLP_N_PARAMS;
constexpr int OW1 = 0, OB1 = OW1 + NH * ND, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NO * NH, OXM = OB4 + NO, OXS = OXM + ND,
              OYM = OXS + ND, OYS = OYM + NO;
static_assert(OXM == NTRAIN, "parameter layout");
static_assert(OYS + NO == NPARAM, "parameter layout");

constexpr int MS = 32;     // samples per CTA
constexpr int AS = 36;     // row stride of activation tiles: 16-B rows, float4 columns conflict-free
constexpr int MT = 256;    // threads per CTA: 8 warps
static_assert(MT / 32 == NO && MS == 32, "output layer maps one warp per output, one lane per sample");

// shared-memory carve (floats)
constexpr int SM_W = NH * (NH + 1), SM_B = NH, SM_X = ND * AS, SM_Z = NH * AS, SM_Y = NO * AS;
constexpr int SM_FLOATS = SM_W + SM_B + SM_X + 4 * SM_Z + SM_Y + 8;
constexpr size_t SM_BYTES = sizeof(float) * SM_FLOATS;

constexpr double kRc = 10.0, kMu0 = 2.0, kMu1 = 10.0, kSig = 0.4;   // descriptors
constexpr double kRphi = 8.0;                                      // support of the correction
constexpr double kPiD = 3.14159265358979323846;

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu_f(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float4 ld4s(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// W [out][in] (global) -> Wsm[j*(IN+1) + i]; biases
template <int IN>
__device__ void stage_w(float *Wsm, float *bsm, const float *W, const float *b, int out) {
    for (int e = threadIdx.x; e < out * IN; e += MT) {
        const int j = e / IN, i = e - j * IN;
        Wsm[j * (IN + 1) + i] = W[e];
    }
    for (int j = threadIdx.x; j < out; j += MT) bsm[j] = b[j];
}

// Z = W A + b, Aout = silu(Z) for a 128-unit layer.  Lane -> units lane + 32 r,
// warp -> samples 4w..4w+3.  Ain may alias Aout: all reads finish before the
// barrier that precedes the writes.
template <int IN>
__device__ void fwd_hidden(const float *Wsm, const float *bsm, const float *Ain, float *Zout, float *Aout) {
    const int lane = threadIdx.x & 31, s0 = (threadIdx.x >> 5) * 4;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float b = bsm[lane + 32 * r];
        acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = b;
    }
#pragma unroll 4
    for (int i = 0; i < IN; ++i) {
        const float4 a = ld4s(Ain + i * AS + s0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float w = Wsm[(lane + 32 * r) * (IN + 1) + i];
            acc[r][0] = fmaf(w, a.x, acc[r][0]);
            acc[r][1] = fmaf(w, a.y, acc[r][1]);
            acc[r][2] = fmaf(w, a.z, acc[r][2]);
            acc[r][3] = fmaf(w, a.w, acc[r][3]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int j = lane + 32 * r;
        float4 z = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        *reinterpret_cast<float4 *>(Zout + j * AS + s0) = z;
        *reinterpret_cast<float4 *>(Aout + j * AS + s0) =
            make_float4(silu_f(z.x), silu_f(z.y), silu_f(z.z), silu_f(z.w));
    }
    __syncthreads();
}

// delta of the previous hidden layer, in place over its pre-activations:
// Zprev[i][s] <- (sum_j W[j][i] Dz[j][s]) * silu'(Zprev[i][s]).  Lane -> units
// lane + 32 r, warp -> samples 4w..4w+3; each thread rewrites its own elements.
template <int OUTN>
__device__ void back_hidden(const float *Wsm, const float *Dz, float *Zprev) {
    const int lane = threadIdx.x & 31, s0 = (threadIdx.x >> 5) * 4;
    float acc[4][4] = {};
#pragma unroll 4
    for (int j = 0; j < OUTN; ++j) {
        const float4 d = ld4s(Dz + j * AS + s0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float w = Wsm[j * (NH + 1) + lane + 32 * r];
            acc[r][0] = fmaf(w, d.x, acc[r][0]);
            acc[r][1] = fmaf(w, d.y, acc[r][1]);
            acc[r][2] = fmaf(w, d.z, acc[r][2]);
            acc[r][3] = fmaf(w, d.w, acc[r][3]);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        float *zp = Zprev + (lane + 32 * r) * AS + s0;
        const float4 z = ld4s(zp);
        *reinterpret_cast<float4 *>(zp) = make_float4(acc[r][0] * dsilu_f(z.x), acc[r][1] * dsilu_f(z.y),
                                                      acc[r][2] * dsilu_f(z.z), acc[r][3] * dsilu_f(z.w));
    }
}

// gW[j][i] = sum_s Dz[j][s] Ain[i][s] (this CTA's samples), gb[j] = sum_s Dz[j][s]
// for a 128 x IN layer.  Lane -> inputs lane + 32 ri, warp -> 16 units.
template <int IN>
__device__ void grad_layer(const float *Dz, const float *Ain, float *gW, float *gb) {
    constexpr int RI = IN / 32;
    const int lane = threadIdx.x & 31, j0 = (threadIdx.x >> 5) * 16;
    float acc[16][RI] = {};
#pragma unroll 1
    for (int s = 0; s < MS; s += 4) {
        float4 a[RI];
#pragma unroll
        for (int ri = 0; ri < RI; ++ri) a[ri] = ld4s(Ain + (lane + 32 * ri) * AS + s);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
            const float4 d = ld4s(Dz + (j0 + jj) * AS + s);
#pragma unroll
            for (int ri = 0; ri < RI; ++ri) acc[jj][ri] += dot4(d, a[ri]);
        }
    }
#pragma unroll
    for (int jj = 0; jj < 16; ++jj)
#pragma unroll
        for (int ri = 0; ri < RI; ++ri) gW[(j0 + jj) * IN + lane + 32 * ri] = acc[jj][ri];
    if (threadIdx.x < NH) {
        float b = 0.0f;
        for (int s = 0; s < MS; ++s) b += Dz[threadIdx.x * AS + s];
        gb[threadIdx.x] = b;
    }
}

__device__ void silu_tile(const float *Z, float *A) {
    for (int e = threadIdx.x; e < NH * MS; e += MT) {
        const int i = e / MS, s = e - i * MS;
        A[i * AS + s] = silu_f(Z[i * AS + s]);
    }
}

// One network pass over samples [32 b, 32 b + 32) of n.  T == nullptr: forward
// only, C = y_mean + y_std y.  Otherwise the loss partial and the gradient
// partials of this CTA go to lpart[b] and gpart[b][.].  tick (optional) is
// advanced by one by CTA 0: the Adam step counter of graph-replayed training.
__global__ void __launch_bounds__(MT, 1)
k_mlp(const float *__restrict__ theta, const float *__restrict__ D, const float *__restrict__ T, int n,
      float *__restrict__ C, float *__restrict__ gpart, float *__restrict__ lpart, int *tick) {
    extern __shared__ __align__(16) float sm[];
    float *Wsm = sm, *bsm = Wsm + SM_W, *X = bsm + SM_B, *Z1 = X + SM_X, *Z2 = Z1 + SM_Z, *Z3 = Z2 + SM_Z,
          *A = Z3 + SM_Z, *Y = A + SM_Z, *red = Y + SM_Y;
    const int tid = threadIdx.x;
    const long long sb = (long long)blockIdx.x * MS;
    const int nv = (int)min((long long)MS, (long long)n - sb);
    if (tick && blockIdx.x == 0 && tid == 0) *tick += 1;

    for (int e = tid; e < ND * MS; e += MT) {
        const int s = e / ND, i = e - s * ND;
        float v = 0.0f;
        if (s < nv) v = (D[(sb + s) * ND + i] - theta[OXM + i]) / theta[OXS + i];
        X[i * AS + s] = v;
    }
    stage_w<ND>(Wsm, bsm, theta + OW1, theta + OB1, NH);
    __syncthreads();
    fwd_hidden<ND>(Wsm, bsm, X, Z1, A);
    stage_w<NH>(Wsm, bsm, theta + OW2, theta + OB2, NH);
    __syncthreads();
    fwd_hidden<NH>(Wsm, bsm, A, Z2, A);
    stage_w<NH>(Wsm, bsm, theta + OW3, theta + OB3, NH);
    __syncthreads();
    fwd_hidden<NH>(Wsm, bsm, A, Z3, A);
    stage_w<NH>(Wsm, bsm, theta + OW4, theta + OB4, NO);
    __syncthreads();
    const int o = tid >> 5, s = tid & 31;
    float y = bsm[o];
#pragma unroll 8
    for (int i = 0; i < NH; ++i) y = fmaf(Wsm[o * (NH + 1) + i], A[i * AS + s], y);
    if (!T) {
        if (s < nv) C[(sb + s) * NO + o] = theta[OYM + o] + theta[OYS + o] * y;
        return;
    }
    // output deltas and the loss
    const float inv = 1.0f / ((float)n * (float)NO);
    float d = 0.0f;
    if (s < nv) d = y - (T[(sb + s) * NO + o] - theta[OYM + o]) / theta[OYS + o];
    float l = d * d;
    for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
    if (s == 0) red[o] = l;
    Y[o * AS + s] = 2.0f * d * inv;
    __syncthreads();
    if (tid == 0) {
        float t = 0.0f;
        for (int w = 0; w < MT / 32; ++w) t += red[w];
        lpart[blockIdx.x] = t * inv;
    }
    float *g = gpart + (size_t)blockIdx.x * NTRAIN;
    // output layer: gW4[o][i] = sum_s dY[o][s] A3[i][s]
    {
        const int i = tid & (NH - 1), o0 = (tid >> 7) * 4;
        float acc[4] = {};
        for (int ss = 0; ss < MS; ss += 4) {
            const float4 a = ld4s(A + i * AS + ss);
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += dot4(ld4s(Y + (o0 + k) * AS + ss), a);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) g[OW4 + (o0 + k) * NH + i] = acc[k];
        if (tid < NO) {
            float b = 0.0f;
            for (int ss = 0; ss < MS; ++ss) b += Y[tid * AS + ss];
            g[OB4 + tid] = b;
        }
    }
    back_hidden<NO>(Wsm, Y, Z3);          // Z3 <- delta of layer 3
    __syncthreads();
    silu_tile(Z2, A);                      // A <- input of layer 3
    stage_w<NH>(Wsm, bsm, theta + OW3, theta + OB3, NH);
    __syncthreads();
    grad_layer<NH>(Z3, A, g + OW3, g + OB3);
    back_hidden<NH>(Wsm, Z3, Z2);         // Z2 <- delta of layer 2
    __syncthreads();
    silu_tile(Z1, A);                      // A <- input of layer 2
    stage_w<NH>(Wsm, bsm, theta + OW2, theta + OB2, NH);
    __syncthreads();
    grad_layer<NH>(Z2, A, g + OW2, g + OB2);
    back_hidden<NH>(Wsm, Z2, Z1);         // Z1 <- delta of layer 1
    __syncthreads();
    grad_layer<ND>(Z1, X, g + OW1, g + OB1);
}

struct AdamP {
    float lr, b1, b2, eps;
};

__device__ __forceinline__ void adam_update(float &th, float &m, float &v, float g, int t, const AdamP &hp) {
    m = hp.b1 * m + (1.0f - hp.b1) * g;
    v = hp.b2 * v + (1.0f - hp.b2) * g * g;
    const float c1 = (float)(1.0 - pow((double)hp.b1, (double)t));
    const float c2 = (float)(1.0 - pow((double)hp.b2, (double)t));
    th -= hp.lr * (m / c1) / (sqrtf(v / c2) + hp.eps);
}

// g[p] = sum over CTAs of the partials (fixed order).  grad (optional) gets g;
// with theta, an Adam step numbered *tick (or t when tick is null).  CTA 0
// sums the loss partials into loss (optional) and loss_hist[step - 1 - t0].
__global__ void k_mlp_reduce(int nblk, const float *__restrict__ gpart, const float *__restrict__ lpart,
                             float *grad, float *loss, float *theta, float *m, float *v, AdamP hp, const int *tick,
                             int t, int t0, float *loss_hist, int hist_len) {
    const int step = tick ? *tick : t;
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        float l = 0.0f;
        for (int b = threadIdx.x; b < nblk; b += 32) l += lpart[b];
        for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
        if (threadIdx.x == 0) {
            if (loss) *loss = l;
            const int h = step - 1 - t0;
            if (loss_hist && h >= 0 && h < hist_len) loss_hist[h] = l;
        }
    }
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NTRAIN) return;
    float gs = 0.0f;
    for (int b = 0; b < nblk; ++b) gs += gpart[(size_t)b * NTRAIN + p];
    if (grad) grad[p] = gs;
    if (theta) adam_update(theta[p], m[p], v[p], gs, step, hp);
}

__global__ void k_adam(float *theta, float *m, float *v, const float *grad, int t, AdamP hp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NTRAIN) adam_update(theta[p], m[p], v[p], grad[p], t, hp);
}

__global__ void k_set_int(int *p, int v) { *p = v; }

// D[I][k]: one block per atom, one thread per descriptor
__global__ void k_descriptors(int n, const double *xyz, const double *Z, float *D) {
    const int I = blockIdx.x, k = threadIdx.x;
    if (I >= n || k >= ND) return;
    const double mu = kMu0 + (kMu1 - kMu0) * k / (ND - 1);
    const double xi = xyz[3 * I], yi = xyz[3 * I + 1], zi = xyz[3 * I + 2];
    double s = 0.0;
    for (int J = 0; J < n; ++J) {
        if (J == I) continue;
        const double dx = xyz[3 * J] - xi, dy = xyz[3 * J + 1] - yi, dz = xyz[3 * J + 2] - zi;
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r >= kRc) continue;
        const double fc = 0.5 * (1.0 + cos(kPiD * r / kRc));
        const double u = r - mu;
        s += Z[J] * exp(-u * u / (2.0 * kSig * kSig)) * fc;
    }
    D[(size_t)I * ND + k] = (float)s;
}

// column statistics: blocks 0..31 the descriptors, 32..39 the targets
__global__ void k_col_stats(int n, const float *D, const float *T, float *theta) {
    __shared__ double red[2][32];
    const int c = blockIdx.x;
    const bool isx = c < ND;
    const float *src = isx ? D + c : T + (c - ND);
    const int ld = isx ? ND : NO;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += src[(size_t)i * ld];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = s;
    __syncthreads();
    double mean = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mean += red[0][w];
    mean /= n;
    double q = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double u = src[(size_t)i * ld] - mean;
        q += u * u;
    }
    for (int off = 16; off > 0; off >>= 1) q += __shfl_down_sync(0xffffffffu, q, off);
    if ((threadIdx.x & 31) == 0) red[1][threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        double var = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) var += red[1][w];
        const double sd = sqrt(var / n);
        if (isx) {
            theta[OXM + c] = (float)mean;
            theta[OXS + c] = (float)fmax(sd, 1e-2);
        } else {
            theta[OYM + c - ND] = (float)mean;
            theta[OYS + c - ND] = (float)fmax(sd, 1e-8);
        }
    }
}

// --- correction basis --------------------------------------------------------
struct Basis {
    double kappa[NO], norm[NO];   // g_j = norm_j exp(-kappa_j r^2)
    double Linv[NO * NO];         // phi_k = sum_j Linv[k][j] g_j
};

Basis make_basis() {
    Basis B{};
    for (int j = 0; j < NO; ++j) {
        B.kappa[j] = 0.5 * std::pow(16.0, j / 7.0);
        B.norm[j] = std::pow(B.kappa[j] / kPiD, 1.5);
    }
    // S_kl = (k_k k_l / (pi (k_k + k_l)))^{3/2}; Cholesky S = L L^T, then L^-1
    double S[NO][NO], L[NO][NO] = {}, Li[NO][NO] = {};
    for (int k = 0; k < NO; ++k)
        for (int l = 0; l < NO; ++l) {
            const double red = B.kappa[k] * B.kappa[l] / (B.kappa[k] + B.kappa[l]);
            S[k][l] = std::pow(red / kPiD, 1.5);
        }
    for (int j = 0; j < NO; ++j) {
        double d = S[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        L[j][j] = std::sqrt(d);
        for (int i = j + 1; i < NO; ++i) {
            double v = S[i][j];
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v / L[j][j];
        }
    }
    for (int c = 0; c < NO; ++c)          // forward substitution, column by column
        for (int i = 0; i < NO; ++i) {
            double v = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[i][k] * Li[k][c];
            Li[i][c] = v / L[i][i];
        }
    for (int k = 0; k < NO; ++k)
        for (int j = 0; j < NO; ++j) B.Linv[k * NO + j] = Li[k][j];
    return B;
}

__device__ __forceinline__ void phi_vals(const Basis &B, double d2, double phi[NO]) {
    double g[NO];
#pragma unroll
    for (int j = 0; j < NO; ++j) g[j] = B.norm[j] * exp(-B.kappa[j] * d2);
#pragma unroll
    for (int k = 0; k < NO; ++k) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NO; ++j) s += B.Linv[k * NO + j] * g[j];
        phi[k] = s;
    }
}

// ceff[I][j] = sum_k c[I][k] Linv[k][j]: coefficients of the raw Gaussians
template <typename T>
__global__ void k_coeff_raw(int natoms, Basis B, const T *c, double *ceff) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= natoms * NO) return;
    const int I = e / NO, j = e - I * NO;
    double s = 0.0;
    for (int k = 0; k < NO; ++k) s += (double)c[I * NO + k] * B.Linv[k * NO + j];
    ceff[e] = s;
}

// one CTA per cell: the atoms within R_PHI of the cell's box, listed in atom
// order by warp 0 (chunks of up to 255), then every Gauss point sums their
// terms; 256 threads x 8 points cover nq^3 <= 2048 (nq <= 12)
constexpr int kListMax = 256;
constexpr int kCorrThreads = 256;
static_assert(EFE_MAXNQ * EFE_MAXNQ * EFE_MAXNQ <= 8 * kCorrThreads, "points per thread");
__global__ void __launch_bounds__(kCorrThreads)
k_correction(MeshDev m, Tables1D T, Basis B, int natoms, const double *__restrict__ atoms,
             const double *__restrict__ ceff, double *__restrict__ out) {
    __shared__ int list[kListMax];
    __shared__ int cnt, next;
    const int c = blockIdx.x;
    const int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
    const double lo[3] = {cx * m.h, cy * m.h, cz * m.h};
    const double R2 = kRphi * kRphi;
    double acc[8];
    const int nqt = (m.nq3 + blockDim.x - 1) / blockDim.x;   // <= 8
    for (int k = 0; k < 8; ++k) acc[k] = 0.0;
    int start = 0;
    while (true) {
        if (threadIdx.x < 32) {
            int n = 0, I0 = start;
            for (; I0 < natoms && n < kListMax - 32; I0 += 32) {
                const int I = I0 + threadIdx.x;
                bool ok = false;
                if (I < natoms) {
                    double d2 = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        const double p = atoms[3 * I + a];
                        const double q = fmin(fmax(p, lo[a]), lo[a] + m.h);
                        d2 += (p - q) * (p - q);
                    }
                    ok = d2 < R2;
                }
                const unsigned mask = __ballot_sync(0xffffffffu, ok);
                if (ok) list[n + __popc(mask & ((1u << threadIdx.x) - 1u))] = I;
                n += __popc(mask);
            }
            if (threadIdx.x == 0) {
                cnt = n;
                next = I0;
            }
        }
        __syncthreads();
        const int n = cnt;
        for (int t = 0; t < nqt && t < 8; ++t) {
            const int q = threadIdx.x + t * blockDim.x;
            if (q >= m.nq3) break;
            double x, y, z;
            quad_point(m, T.xq, c, q, x, y, z);
            double s = 0.0;
            for (int l = 0; l < n; ++l) {
                const int I = list[l];
                const double dx = x - atoms[3 * I], dy = y - atoms[3 * I + 1], dz = z - atoms[3 * I + 2];
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 >= R2) continue;
                const double *ce = ceff + (size_t)I * NO;
#pragma unroll
                for (int j = 0; j < NO; ++j) s += ce[j] * B.norm[j] * exp(-B.kappa[j] * d2);
            }
            acc[t] += s;
        }
        const int nx = next;
        __syncthreads();
        if (nx >= natoms) break;
        start = nx;
    }
    for (int t = 0; t < nqt && t < 8; ++t) {
        const int q = threadIdx.x + t * blockDim.x;
        if (q < m.nq3) out[(size_t)c * m.nq3 + q] = acc[t];
    }
}

// cells of the box [R - R_PHI, R + R_PHI] clipped to the mesh
__device__ __forceinline__ void support_cells(const MeshDev &m, const double *R, int lo[3], int hi[3]) {
    const int nc[3] = {m.nx, m.ny, m.nz};
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(0, (int)floor((R[a] - kRphi) / m.h));
        hi[a] = min(nc[a] - 1, (int)floor((R[a] + kRphi) / m.h));
    }
}

template <int NV>
__device__ void block_sum(double (&v)[NV], double *red, double *out) {
    // red: (blockDim/32) x NV doubles
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = v[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) red[w * NV + k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NV; k += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += red[i * NV + k];
        out[k] = s;
    }
}

// r[I][k] = sum_q w_q (rho - base)(x_q) phi_k(|x_q - R_I|): one CTA per atom
__global__ void __launch_bounds__(128)
k_fit_rhs(MeshDev m, Tables1D T, Basis B, const double *__restrict__ atoms, const double *__restrict__ rho,
          const double *__restrict__ base, double *__restrict__ r) {
    __shared__ double red[4 * NO];
    const int I = blockIdx.x;
    const double R[3] = {atoms[3 * I], atoms[3 * I + 1], atoms[3 * I + 2]};
    int lo[3], hi[3];
    support_cells(m, R, lo, hi);
    const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
    const long long npts = (long long)ex * ey * ez * m.nq3;
    const double J = 0.125 * m.h * m.h * m.h;
    double acc[NO] = {};
    for (long long e = threadIdx.x; e < npts; e += blockDim.x) {
        const int q = (int)(e % m.nq3);
        const long long cl = e / m.nq3;
        const int c = ((int)(cl / ((long long)ex * ey)) + lo[2]) * m.nx * m.ny +
                      ((int)((cl / ex) % ey) + lo[1]) * m.nx + (int)(cl % ex) + lo[0];
        double x, y, z;
        quad_point(m, T.xq, c, q, x, y, z);
        const double d2 = (x - R[0]) * (x - R[0]) + (y - R[1]) * (y - R[1]) + (z - R[2]) * (z - R[2]);
        if (d2 >= kRphi * kRphi) continue;
        const int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        const size_t gi = (size_t)c * m.nq3 + q;
        const double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J * (base ? rho[gi] - base[gi] : rho[gi]);
        double phi[NO];
        phi_vals(B, d2, phi);
#pragma unroll
        for (int k = 0; k < NO; ++k) acc[k] += w * phi[k];
    }
    block_sum<NO>(acc, red, r + (size_t)I * NO);
}

// A[(I,k),(J,l)] = sum_q w_q phi_Ik phi_Jl over the common support of a pair
// I <= J (one CTA per listed pair), written to both triangles
__global__ void __launch_bounds__(128)
k_fit_gram(MeshDev m, Tables1D T, Basis B, const double *__restrict__ atoms, const int2 *__restrict__ pairs,
           int natoms, double *__restrict__ A) {
    __shared__ double red[4 * NO * NO];
    __shared__ double blk[NO * NO];
    const int2 pr = pairs[blockIdx.x];
    const double RI[3] = {atoms[3 * pr.x], atoms[3 * pr.x + 1], atoms[3 * pr.x + 2]};
    const double RJ[3] = {atoms[3 * pr.y], atoms[3 * pr.y + 1], atoms[3 * pr.y + 2]};
    int loI[3], hiI[3], loJ[3], hiJ[3], lo[3], hi[3];
    support_cells(m, RI, loI, hiI);
    support_cells(m, RJ, loJ, hiJ);
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(loI[a], loJ[a]);
        hi[a] = min(hiI[a], hiJ[a]);
    }
    double acc[NO * NO] = {};
    if (hi[0] >= lo[0] && hi[1] >= lo[1] && hi[2] >= lo[2]) {
        const int ex = hi[0] - lo[0] + 1, ey = hi[1] - lo[1] + 1, ez = hi[2] - lo[2] + 1;
        const long long npts = (long long)ex * ey * ez * m.nq3;
        const double J = 0.125 * m.h * m.h * m.h;
        const double R2 = kRphi * kRphi;
        for (long long e = threadIdx.x; e < npts; e += blockDim.x) {
            const int q = (int)(e % m.nq3);
            const long long cl = e / m.nq3;
            const int c = ((int)(cl / ((long long)ex * ey)) + lo[2]) * m.nx * m.ny +
                          ((int)((cl / ex) % ey) + lo[1]) * m.nx + (int)(cl % ex) + lo[0];
            double x, y, z;
            quad_point(m, T.xq, c, q, x, y, z);
            const double dI = (x - RI[0]) * (x - RI[0]) + (y - RI[1]) * (y - RI[1]) + (z - RI[2]) * (z - RI[2]);
            const double dJ = (x - RJ[0]) * (x - RJ[0]) + (y - RJ[1]) * (y - RJ[1]) + (z - RJ[2]) * (z - RJ[2]);
            if (dI >= R2 || dJ >= R2) continue;
            const int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
            const double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J;
            double pI[NO], pJ[NO];
            phi_vals(B, dI, pI);
            phi_vals(B, dJ, pJ);
#pragma unroll
            for (int k = 0; k < NO; ++k) {
                const double wk = w * pI[k];
#pragma unroll
                for (int l = 0; l < NO; ++l) acc[k * NO + l] += wk * pJ[l];
            }
        }
    }
    block_sum<NO * NO>(acc, red, blk);
    __syncthreads();
    const size_t n8 = (size_t)natoms * NO;
    for (int e = threadIdx.x; e < NO * NO; e += blockDim.x) {
        const int k = e / NO, l = e - k * NO;
        A[(pr.x * NO + k) * n8 + pr.y * NO + l] = blk[e];
        A[(pr.y * NO + l) * n8 + pr.x * NO + k] = blk[e];
    }
}

__global__ void k_add_diag(int n, double v, double *A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) A[(size_t)i * n + i] += v;
}

// max(a + b, 0), keeping non-finite values (fmax would turn a NaN into 0) so
// that the integral test sees them
__global__ void k_clip_sum(long long n, const double *a, const double *b, double *out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        const double v = a[i] + b[i];
        out[i] = isfinite(v) ? fmax(v, 0.0) : v;
    }
}

__global__ void k_scale_into(long long n, double s, const double *a, double *out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = s * a[i];
}

inline unsigned nbl(long long n, int b) { return (unsigned)((n + b - 1) / b); }

thread_local std::string g_mlp_create_err;

// device buffers freed (after the stream drains) when the scope ends
struct Scratch {
    cudaStream_t s;
    std::vector<void *> p;
    explicit Scratch(cudaStream_t st) : s(st) {}
    ~Scratch() {
        if (!p.empty()) cudaStreamSynchronize(s);
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    T *get(size_t n) {
        void *q = nullptr;
        if (cudaMalloc(&q, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return static_cast<T *>(q);
    }
};

}  // namespace

struct efe_mlp {
    std::string err;
    cudaStream_t user = nullptr;
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    int max_n = 0, max_blk = 0;
    float *d_gpart = nullptr, *d_lpart = nullptr, *d_loss = nullptr;
    int *d_tick = nullptr;
};

#define MLP_CUDA(mlp, call)                                                          \
    do {                                                                             \
        cudaError_t _e = (call);                                                     \
        if (_e != cudaSuccess) {                                                     \
            (mlp)->err = std::string(#call) + ": " + cudaGetErrorString(_e);         \
            return EFE_ERR_CUDA;                                                     \
        }                                                                            \
    } while (0)
#define MLP_ARG(mlp, cond, msg)                                                      \
    do {                                                                             \
        if (!(cond)) {                                                               \
            (mlp)->err = msg;                                                        \
            return EFE_ERR_ARG;                                                      \
        }                                                                            \
    } while (0)

static efe_status mlp_launch_check(efe_mlp *mlp, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mlp->err = std::string(what) + ": " + cudaGetErrorString(e);
        return EFE_ERR_CUDA;
    }
    return EFE_OK;
}

static efe_status mlp_pass(efe_mlp *mlp, cudaStream_t s, const float *theta, const float *D, const float *T, int n,
                           float *C, int *tick) {
    static bool attr = false;
    if (!attr) {
        MLP_CUDA(mlp, cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES));
        attr = true;
    }
    const unsigned nb = nbl(n, MS);
    k_mlp<<<nb, MT, SM_BYTES, s>>>(theta, D, T, n, C, mlp->d_gpart, mlp->d_lpart, tick);
    return mlp_launch_check(mlp, "k_mlp");
}

extern "C" {

efe_status efe_mlp_create(void *stream, int max_samples, efe_mlp **out) {
    g_mlp_create_err.clear();
    if (!out || max_samples < 1) {
        g_mlp_create_err = "efe_mlp_create: null output or max_samples < 1";
        return EFE_ERR_ARG;
    }
    *out = nullptr;
    efe_mlp *mlp = new efe_mlp();
    mlp->user = (cudaStream_t)stream;
    mlp->max_n = max_samples;
    mlp->max_blk = (int)nbl(max_samples, MS);
    bool ok = cudaStreamCreateWithFlags(&mlp->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&mlp->ev_a, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&mlp->ev_b, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc((void **)&mlp->d_gpart, sizeof(float) * (size_t)mlp->max_blk * NTRAIN) == cudaSuccess &&
              cudaMalloc((void **)&mlp->d_lpart, sizeof(float) * mlp->max_blk) == cudaSuccess &&
              cudaMalloc((void **)&mlp->d_loss, sizeof(float)) == cudaSuccess &&
              cudaMalloc((void **)&mlp->d_tick, sizeof(int)) == cudaSuccess;
    if (!ok) {
        g_mlp_create_err = std::string("efe_mlp_create: ") + cudaGetErrorString(cudaGetLastError());
        efe_mlp_destroy(mlp);
        return EFE_ERR_OOM;
    }
    *out = mlp;
    return EFE_OK;
}

void efe_mlp_destroy(efe_mlp *mlp) {
    if (!mlp) return;
    if (mlp->user) cudaStreamSynchronize(mlp->user);
    if (mlp->cap) cudaStreamSynchronize(mlp->cap);
    cudaFree(mlp->d_gpart);
    cudaFree(mlp->d_lpart);
    cudaFree(mlp->d_loss);
    cudaFree(mlp->d_tick);
    if (mlp->ev_a) cudaEventDestroy(mlp->ev_a);
    if (mlp->ev_b) cudaEventDestroy(mlp->ev_b);
    if (mlp->cap) cudaStreamDestroy(mlp->cap);
    delete mlp;
}

const char *efe_mlp_last_error(const efe_mlp *mlp) { return mlp ? mlp->err.c_str() : g_mlp_create_err.c_str(); }

efe_status efe_descriptors(efe_mlp *mlp, const double *xyz, const double *zval, int n, float *D) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, n >= 0 && (n == 0 || (xyz && zval && D)), "efe_descriptors: null pointer or n < 0");
    if (n == 0) return EFE_OK;
    k_descriptors<<<n, ND, 0, mlp->user>>>(n, xyz, zval, D);
    return mlp_launch_check(mlp, "k_descriptors");
}

efe_status efe_mlp_forward(efe_mlp *mlp, const float *theta, const float *D, int n, float *C) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, n >= 0 && (n == 0 || (theta && D && C)), "efe_mlp_forward: null pointer or n < 0");
    if (n == 0) return EFE_OK;
    return mlp_pass(mlp, mlp->user, theta, D, nullptr, n, C, nullptr);
}

efe_status efe_mlp_normalise(efe_mlp *mlp, float *theta, const float *D, const float *T, int n) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, theta && D && T && n >= 1, "efe_mlp_normalise: null pointer or n < 1");
    k_col_stats<<<ND + NO, 256, 0, mlp->user>>>(n, D, T, theta);
    return mlp_launch_check(mlp, "k_col_stats");
}

efe_status efe_mlp_loss_grad(efe_mlp *mlp, const float *theta, const float *D, const float *T, int n, float *grad,
                             double *loss) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, theta && D && T && grad && n >= 1, "efe_mlp_loss_grad: null pointer or n < 1");
    MLP_ARG(mlp, n <= mlp->max_n, "efe_mlp_loss_grad: n exceeds the workspace's max_samples");
    EFE_TRY(mlp_pass(mlp, mlp->user, theta, D, T, n, nullptr, nullptr));
    const int nb = (int)nbl(n, MS);
    k_mlp_reduce<<<nbl(NTRAIN, 256), 256, 0, mlp->user>>>(nb, mlp->d_gpart, mlp->d_lpart, grad, mlp->d_loss,
                                                         nullptr, nullptr, nullptr, AdamP{}, nullptr, 1, 0, nullptr,
                                                         0);
    EFE_TRY(mlp_launch_check(mlp, "k_mlp_reduce"));
    if (loss) {
        float l = 0.0f;
        MLP_CUDA(mlp, cudaMemcpyAsync(&l, mlp->d_loss, sizeof(float), cudaMemcpyDeviceToHost, mlp->user));
        MLP_CUDA(mlp, cudaStreamSynchronize(mlp->user));
        *loss = l;
    }
    return EFE_OK;
}

efe_status efe_mlp_adam(efe_mlp *mlp, float *theta, float *m, float *v, const float *grad, int t,
                        const efe_adam *hp) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, theta && m && v && grad && hp && t >= 1, "efe_mlp_adam: null pointer or t < 1");
    k_adam<<<nbl(NTRAIN, 256), 256, 0, mlp->user>>>(theta, m, v, grad, t,
                                                    AdamP{hp->lr, hp->beta1, hp->beta2, hp->eps});
    return mlp_launch_check(mlp, "k_adam");
}

efe_status efe_mlp_train(efe_mlp *mlp, float *theta, float *m, float *v, const float *D, const float *T, int n,
                         int steps, int t0, const efe_adam *hp, float *loss_hist) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, theta && m && v && D && T && hp && n >= 1 && steps >= 0 && t0 >= 0,
            "efe_mlp_train: null pointer, n < 1, steps < 0 or t0 < 0");
    MLP_ARG(mlp, n <= mlp->max_n, "efe_mlp_train: n exceeds the workspace's max_samples");
    if (steps == 0) return EFE_OK;
    // make sure the kernel attribute is set outside the capture
    static bool attr = false;
    if (!attr) {
        MLP_CUDA(mlp, cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES));
        attr = true;
    }
    const int nb = (int)nbl(n, MS);
    const AdamP ap{hp->lr, hp->beta1, hp->beta2, hp->eps};
    cudaStream_t cs = mlp->cap;
    MLP_CUDA(mlp, cudaEventRecord(mlp->ev_a, mlp->user));
    MLP_CUDA(mlp, cudaStreamWaitEvent(cs, mlp->ev_a, 0));
    k_set_int<<<1, 1, 0, cs>>>(mlp->d_tick, t0);
    EFE_TRY(mlp_launch_check(mlp, "k_set_int"));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MLP_CUDA(mlp, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    k_mlp<<<nb, MT, SM_BYTES, cs>>>(theta, D, T, n, nullptr, mlp->d_gpart, mlp->d_lpart, mlp->d_tick);
    k_mlp_reduce<<<nbl(NTRAIN, 256), 256, 0, cs>>>(nb, mlp->d_gpart, mlp->d_lpart, nullptr, nullptr, theta, m, v, ap,
                                                  mlp->d_tick, 0, t0, loss_hist, steps);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess || !graph) {
        mlp->err = std::string("efe_mlp_train: graph capture failed: ") + cudaGetErrorString(ce);
        cudaGetLastError();
        return EFE_ERR_CUDA;
    }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        mlp->err = std::string("efe_mlp_train: graph instantiation failed: ") + cudaGetErrorString(ce);
        return EFE_ERR_CUDA;
    }
    efe_status st = EFE_OK;
    for (int s = 0; s < steps && st == EFE_OK; ++s) {
        ce = cudaGraphLaunch(exec, cs);
        if (ce != cudaSuccess) {
            mlp->err = std::string("efe_mlp_train: cudaGraphLaunch: ") + cudaGetErrorString(ce);
            st = EFE_ERR_CUDA;
        }
    }
    cudaEventRecord(mlp->ev_b, cs);
    cudaStreamWaitEvent(mlp->user, mlp->ev_b, 0);
    cudaStreamSynchronize(cs);
    cudaGraphExecDestroy(exec);
    return st;
}

// The file layout is defined little-endian; the hosts this builds for (x86-64,
// AArch64) are little-endian, so the bytes are written as they are in memory.
static const char kMlpTag[8] = {'E', 'F', 'E', 'M', 'L', 'P', '0', '1'};

efe_status efe_mlp_save(efe_mlp *mlp, const float *theta, const char *path) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, theta && path, "efe_mlp_save: null pointer");
    std::vector<float> h(NPARAM);
    MLP_CUDA(mlp, cudaMemcpyAsync(h.data(), theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, mlp->user));
    MLP_CUDA(mlp, cudaStreamSynchronize(mlp->user));
    FILE *f = std::fopen(path, "wb");
    MLP_ARG(mlp, f != nullptr, std::string("efe_mlp_save: cannot open ") + path);
    const int32_t cnt = NPARAM;
    const bool ok = std::fwrite(kMlpTag, 1, 8, f) == 8 && std::fwrite(&cnt, 4, 1, f) == 1 &&
                    std::fwrite(h.data(), sizeof(float), NPARAM, f) == (size_t)NPARAM;
    const bool closed = std::fclose(f) == 0;
    MLP_ARG(mlp, ok && closed, std::string("efe_mlp_save: write failed for ") + path);
    return EFE_OK;
}

efe_status efe_mlp_load(efe_mlp *mlp, const char *path, float *theta) {
    if (!mlp) return EFE_ERR_ARG;
    MLP_ARG(mlp, theta && path, "efe_mlp_load: null pointer");
    FILE *f = std::fopen(path, "rb");
    MLP_ARG(mlp, f != nullptr, std::string("efe_mlp_load: cannot open ") + path);
    char tag[8];
    int32_t cnt = 0;
    std::vector<float> h(NPARAM);
    const bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kMlpTag, 8) == 0 &&
                    std::fread(&cnt, 4, 1, f) == 1 && cnt == NPARAM &&
                    std::fread(h.data(), sizeof(float), NPARAM, f) == (size_t)NPARAM;
    std::fclose(f);
    MLP_ARG(mlp, ok, std::string("efe_mlp_load: not a parameter file of this network: ") + path);
    MLP_CUDA(mlp, cudaMemcpyAsync(theta, h.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice, mlp->user));
    MLP_CUDA(mlp, cudaStreamSynchronize(mlp->user));
    return EFE_OK;
}

efe_status efe_density_correction(efe_ctx *ctx, const double *c, double *drho_q) {
    if (!ctx) return EFE_ERR_ARG;
    if (!c || !drho_q) {
        ctx->err = "efe_density_correction: null pointer";
        return EFE_ERR_ARG;
    }
    Scratch sc(ctx->stream);
    double *ceff = sc.get<double>((size_t)ctx->natoms * NO);
    if (!ceff) return EFE_ERR_OOM;
    const Basis B = make_basis();
    k_coeff_raw<double><<<nbl((long long)ctx->natoms * NO, 128), 128, 0, ctx->stream>>>(ctx->natoms, B, c, ceff);
    EFE_TRY(efe_check_launch(ctx, "k_coeff_raw"));
    const long long ncell = (long long)ctx->m.nx * ctx->m.ny * ctx->m.nz;
    k_correction<<<(unsigned)ncell, kCorrThreads, 0, ctx->stream>>>(ctx->m, make_tables(ctx), B, ctx->natoms, ctx->d_atoms,
                                                          ceff, drho_q);
    EFE_TRY(efe_check_launch(ctx, "k_correction"));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

efe_status efe_fit_correction(efe_ctx *ctx, const double *rho_q, const double *base_q, double ridge, double *c) {
    if (!ctx) return EFE_ERR_ARG;
    if (!rho_q || !c || !(ridge >= 0.0)) {
        ctx->err = "efe_fit_correction: null pointer or ridge < 0";
        return EFE_ERR_ARG;
    }
    const int na = ctx->natoms;
    const int n8 = na * NO;
    std::vector<int2> pairs;
    for (int I = 0; I < na; ++I)
        for (int J = I; J < na; ++J) {
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                const double u = ctx->xyz[3 * I + a] - ctx->xyz[3 * J + a];
                d2 += u * u;
            }
            if (d2 < 4.0 * kRphi * kRphi) pairs.push_back(make_int2(I, J));
        }
    Scratch sc(ctx->stream);
    double *A = sc.get<double>((size_t)n8 * n8);
    int2 *dp = sc.get<int2>(pairs.size());
    int *info = sc.get<int>(1);
    if (!A || !dp || !info) return EFE_ERR_OOM;
    EFE_CUDA(ctx, cudaMemcpyAsync(dp, pairs.data(), sizeof(int2) * pairs.size(), cudaMemcpyHostToDevice, ctx->stream));
    EFE_CUDA(ctx, cudaMemsetAsync(A, 0, sizeof(double) * (size_t)n8 * n8, ctx->stream));
    const Basis B = make_basis();
    const Tables1D T = make_tables(ctx);
    k_fit_rhs<<<na, 128, 0, ctx->stream>>>(ctx->m, T, B, ctx->d_atoms, rho_q, base_q, c);
    EFE_TRY(efe_check_launch(ctx, "k_fit_rhs"));
    k_fit_gram<<<(unsigned)pairs.size(), 128, 0, ctx->stream>>>(ctx->m, T, B, ctx->d_atoms, dp, na, A);
    EFE_TRY(efe_check_launch(ctx, "k_fit_gram"));
    if (ridge > 0.0) k_add_diag<<<nbl(n8, 128), 128, 0, ctx->stream>>>(n8, ridge, A);
    if (cusolverDnSetStream(ctx->solver, ctx->stream) != CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnSetStream failed";
        return EFE_ERR_CUDA;
    }
    int lwork = 0;
    if (cusolverDnDpotrf_bufferSize(ctx->solver, CUBLAS_FILL_MODE_UPPER, n8, A, n8, &lwork) !=
        CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnDpotrf_bufferSize failed";
        return EFE_ERR_CUDA;
    }
    double *work = sc.get<double>((size_t)lwork);
    if (!work) return EFE_ERR_OOM;
    // A is symmetric, so its row-major storage is also its column-major storage
    if (cusolverDnDpotrf(ctx->solver, CUBLAS_FILL_MODE_UPPER, n8, A, n8, work, lwork, info) !=
        CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnDpotrf failed";
        return EFE_ERR_CUDA;
    }
    int hinfo = 0;
    EFE_CUDA(ctx, cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hinfo != 0) {
        ctx->err = "efe_fit_correction: normal equations not positive definite (potrf info " +
                   std::to_string(hinfo) + "); use ridge > 0";
        return EFE_ERR_NOT_SPD;
    }
    if (cusolverDnDpotrs(ctx->solver, CUBLAS_FILL_MODE_UPPER, n8, 1, A, n8, c, n8, info) != CUSOLVER_STATUS_SUCCESS) {
        ctx->err = "cusolverDnDpotrs failed";
        return EFE_ERR_CUDA;
    }
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

}  // extern "C"

namespace {

// rho_q <- max(rho_sup + drho(c), 0) scaled to N_e, rho_sup already in rho_q;
// c (natoms x 8, float or double) in the orthonormal basis.  *ok = false (rho_q
// untouched) when the corrected density is not finite or has no charge.
template <typename T>
efe_status corrected_density(efe_ctx *ctx, const T *c, double *rho_q, bool *ok) {
    *ok = false;
    const int na = ctx->natoms;
    const long long nq = ctx->n_quad;
    Scratch sc(ctx->stream);
    double *ceff = sc.get<double>((size_t)na * NO);
    double *rho = sc.get<double>(nq);
    if (!ceff || !rho) return EFE_ERR_OOM;
    const Basis B = make_basis();
    k_coeff_raw<T><<<nbl((long long)na * NO, 128), 128, 0, ctx->stream>>>(na, B, c, ceff);
    EFE_TRY(efe_check_launch(ctx, "k_coeff_raw"));
    const long long ncell = (long long)ctx->m.nx * ctx->m.ny * ctx->m.nz;
    k_correction<<<(unsigned)ncell, kCorrThreads, 0, ctx->stream>>>(ctx->m, make_tables(ctx), B, na, ctx->d_atoms,
                                                                  ceff, rho);
    EFE_TRY(efe_check_launch(ctx, "k_correction"));
    k_clip_sum<<<nbl(nq, 256), 256, 0, ctx->stream>>>(nq, rho_q, rho, rho);
    double tot = 0.0;
    EFE_TRY(efe_integrate(ctx, rho, nullptr, &tot));
    double ne = 0.0;
    for (double z : ctx->zval) ne += z;
    if (!std::isfinite(tot) || !(tot > 0.0)) return EFE_OK;      // the superposition stays in rho_q
    k_scale_into<<<nbl(nq, 256), 256, 0, ctx->stream>>>(nq, ne / tot, rho, rho_q);
    EFE_TRY(efe_check_launch(ctx, "k_scale_into"));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *ok = true;
    return EFE_OK;
}

}  // namespace

extern "C" {

efe_status efe_corrected_density(efe_ctx *ctx, const double *c, double kappa, double *rho_q, int *fallback) {
    if (!ctx) return EFE_ERR_ARG;
    if (!c || !rho_q || !(kappa > 0.0)) {
        ctx->err = "efe_corrected_density: null pointer or kappa <= 0";
        return EFE_ERR_ARG;
    }
    if (fallback) *fallback = 1;
    EFE_TRY(efe_atomic_density(ctx, kappa, rho_q));
    bool ok = false;
    EFE_TRY(corrected_density<double>(ctx, c, rho_q, &ok));
    if (fallback) *fallback = ok ? 0 : 1;
    return EFE_OK;
}

efe_status efe_warm_start(efe_ctx *ctx, efe_mlp *mlp, const float *theta, double kappa, double *rho_q,
                          int *fallback) {
    if (!ctx) return EFE_ERR_ARG;
    if (!rho_q || !(kappa > 0.0) || (theta && !mlp)) {
        ctx->err = "efe_warm_start: null rho_q, kappa <= 0, or parameters without a workspace";
        return EFE_ERR_ARG;
    }
    if (fallback) *fallback = 1;
    EFE_TRY(efe_atomic_density(ctx, kappa, rho_q));
    if (!theta) return EFE_OK;
    const int na = ctx->natoms;
    Scratch sc(ctx->stream);
    double *dz = sc.get<double>(na);
    float *D = sc.get<float>((size_t)na * ND);
    float *C = sc.get<float>((size_t)na * NO);
    if (!dz || !D || !C) return EFE_ERR_OOM;
    EFE_CUDA(ctx, cudaMemcpyAsync(dz, ctx->zval.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
    k_descriptors<<<na, ND, 0, ctx->stream>>>(na, ctx->d_atoms, dz, D);
    EFE_TRY(efe_check_launch(ctx, "k_descriptors"));
    static bool attr = false;
    if (!attr) {
        EFE_CUDA(ctx, cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_BYTES));
        attr = true;
    }
    k_mlp<<<nbl(na, MS), MT, SM_BYTES, ctx->stream>>>(theta, D, nullptr, na, C, nullptr, nullptr, nullptr);
    EFE_TRY(efe_check_launch(ctx, "k_mlp"));
    bool ok = false;
    EFE_TRY(corrected_density<float>(ctx, C, rho_q, &ok));
    if (fallback) *fallback = ok ? 0 : 1;
    return EFE_OK;
}

}  // extern "C"
