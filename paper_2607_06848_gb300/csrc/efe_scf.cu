// Self-consistent field machinery on the GPU (paper Sec. II.A, Sec. IV):
// density at the quadrature points (Eq. rhocompute), Fermi level (Eq.
// electronconstraint) at 500 K, LDA exchange-correlation in the Perdew-Wang
// form, the electrostatic potential of rho + b_sm by FE conjugate gradients
// (Eqs. EellocReform, poisson), energies, Anderson mixing, and the SCF loop.
#include "efe_internal.cuh"
#include "efe_funcs.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace {

inline unsigned nb(long long n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ inline bool interior_node(const MeshDev &m, int ix, int iy, int iz) {
    return ix > 0 && iy > 0 && iz > 0 && ix < m.Gx - 1 && iy < m.Gy - 1 && iz < m.Gz - 1;
}

// ---------------------------------------------------------------------------
// psi(x_q) = sum_l N_l(x_q) U[node(c,l)] + sum_{pairs of c} sum_f a_f(x_q) Ue[4I+f]
// per cell by sum factorisation (three 1-D contractions with B1), columns in
// tiles of TJ.  mode 0: rho[q] += sum_j w2[j] psi_j(q)^2; mode 1: out[q] = psi_0(q).
// ---------------------------------------------------------------------------
constexpr int TJ = 8;

__global__ void k_cell_values(MeshDev m, Tables1D T, const double *U, const double *Ue, int N,
                              const int *cell_pair_ptr, const int *cell_pair_idx, const int *pair_atom,
                              const double *pair_avals, const double *w2, int mode, double *out) {
    extern __shared__ double sh[];
    const int np1 = m.np1, nq = m.nq, ne = m.ne, nq3 = m.nq3;
    double *su = sh;                          // ne x TJ
    double *t1 = su + ne * TJ;                // np1*np1*nq
    double *t2 = t1 + np1 * np1 * nq;         // np1*nq*nq
    double *sB = t2 + np1 * nq * nq;          // nq*np1
    const int c = blockIdx.x;
    const int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
    for (int i = threadIdx.x; i < nq * np1; i += blockDim.x) sB[i] = T.B1[i];
    double acc[4] = {0, 0, 0, 0};               // per thread: points q = tid + k*blockDim (nq3 <= 1024)
    const int p0 = cell_pair_ptr ? cell_pair_ptr[c] : 0, p1 = cell_pair_ptr ? cell_pair_ptr[c + 1] : 0;
    for (int j0 = 0; j0 < N; j0 += TJ) {
        __syncthreads();
        for (int i = threadIdx.x; i < ne * TJ; i += blockDim.x) {
            const int l = i / TJ, jj = i % TJ;
            const int lx = l % np1, ly = (l / np1) % np1, lz = l / (np1 * np1);
            const long long node = ((long long)(cz * m.p + lz) * m.Gy + (cy * m.p + ly)) * m.Gx + (cx * m.p + lx);
            su[i] = (j0 + jj < N) ? U[node * N + j0 + jj] : 0.0;
        }
        for (int jj = 0; jj < TJ && j0 + jj < N; ++jj) {
            __syncthreads();
            // t1[az][ay][qx] = sum_ax B1[qx][ax] u[az][ay][ax]
            for (int i = threadIdx.x; i < np1 * np1 * nq; i += blockDim.x) {
                const int qx = i % nq, zy = i / nq;
                double s = 0.0;
                for (int ax = 0; ax < np1; ++ax) s += sB[qx * np1 + ax] * su[(zy * np1 + ax) * TJ + jj];
                t1[i] = s;
            }
            __syncthreads();
            // t2[az][qy][qx] = sum_ay B1[qy][ay] t1[az][ay][qx]
            for (int i = threadIdx.x; i < np1 * nq * nq; i += blockDim.x) {
                const int qx = i % nq, qy = (i / nq) % nq, az = i / (nq * nq);
                double s = 0.0;
                for (int ay = 0; ay < np1; ++ay) s += sB[qy * np1 + ay] * t1[(az * np1 + ay) * nq + qx];
                t2[i] = s;
            }
            __syncthreads();
            int k = 0;
            for (int q = threadIdx.x; q < nq3; q += blockDim.x, ++k) {
                const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
                double s = 0.0;
                for (int az = 0; az < np1; ++az) s += sB[qz * np1 + az] * t2[(az * nq + qy) * nq + qx];
                for (int pp = p0; pp < p1; ++pp) {
                    const int pr = cell_pair_idx[pp];
                    const int I = pair_atom[pr];
                    const double *av = pair_avals + (size_t)pr * 4 * nq3;
                    for (int f = 0; f < 4; ++f) s += av[f * nq3 + q] * Ue[(size_t)(4 * I + f) * N + j0 + jj];
                }
                if (mode == 0) acc[k] += w2[j0 + jj] * s * s;
                else out[(size_t)c * nq3 + q] = s;
            }
        }
    }
    if (mode == 0) {
        int k = 0;
        for (int q = threadIdx.x; q < nq3; q += blockDim.x, ++k) out[(size_t)c * nq3 + q] = acc[k];
    }
}

// Enrichment values a_f at the quadrature points of every (atom, cell) pair.
__global__ void k_pair_values(MeshDev m, Tables1D T, FuncParams fp, const PairInfo *pairs, const double *atoms,
                              double *avals) {
    const PairInfo pr = pairs[blockIdx.x];
    const double ax = atoms[3 * pr.atom], ay = atoms[3 * pr.atom + 1], az = atoms[3 * pr.atom + 2];
    for (int q = threadIdx.x; q < m.nq3; q += blockDim.x) {
        double x, y, z;
        quad_point(m, T.xq, pr.cell, q, x, y, z);
        double a[4], ga[4][3], b[4];
        FuncParams f2 = fp;
        f2.nonlocal = 0;
        eval_funcs(f2, x - ax, y - ay, z - az, a, ga, b);
        for (int f = 0; f < 4; ++f) avals[((size_t)blockIdx.x * 4 + f) * m.nq3 + q] = a[f];
    }
}

// F_j += sum_q w_q J N_j(x_q) f(x_q) for the cells of one colour (no atomics).
__global__ void k_project_colour(MeshDev m, Tables1D T, int colour, const double *fq, double *F) {
    extern __shared__ double sh[];
    const int np1 = m.np1, nq = m.nq, nq3 = m.nq3;
    double *g = sh;                   // nq3
    double *t2 = g + nq3;             // nq*nq*np1   [qz][qy][ax]
    double *t1 = t2 + nq * nq * np1;  // nq*np1*np1  [qz][ay][ax]
    const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
    const int hx = (m.nx - ox + 1) / 2, hy = (m.ny - oy + 1) / 2;
    const int b = blockIdx.x;
    const int cx = 2 * (b % hx) + ox, cy = 2 * ((b / hx) % hy) + oy, cz = 2 * (b / (hx * hy)) + oz;
    const int c = (cz * m.ny + cy) * m.nx + cx;
    const double J = 0.125 * m.h * m.h * m.h;
    for (int q = threadIdx.x; q < nq3; q += blockDim.x) {
        const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
        g[q] = T.wq[qx] * T.wq[qy] * T.wq[qz] * J * fq[(size_t)c * nq3 + q];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nq * nq * np1; i += blockDim.x) {
        const int ax = i % np1, qy = (i / np1) % nq, qz = i / (np1 * nq);
        double s = 0.0;
        for (int qx = 0; qx < nq; ++qx) s += T.B1[qx * np1 + ax] * g[(qz * nq + qy) * nq + qx];
        t2[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nq * np1 * np1; i += blockDim.x) {
        const int ax = i % np1, ay = (i / np1) % np1, qz = i / (np1 * np1);
        double s = 0.0;
        for (int qy = 0; qy < nq; ++qy) s += T.B1[qy * np1 + ay] * t2[(qz * nq + qy) * np1 + ax];
        t1[i] = s;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < m.ne; l += blockDim.x) {
        const int ax = l % np1, ay = (l / np1) % np1, az = l / (np1 * np1);
        double s = 0.0;
        for (int qz = 0; qz < nq; ++qz) s += T.B1[qz * np1 + az] * t1[(qz * np1 + ay) * np1 + ax];
        const int ix = cx * m.p + ax, iy = cy * m.p + ay, iz = cz * m.p + az;
        if (!interior_node(m, ix, iy, iz)) continue;
        F[((long long)iz * m.Gy + iy) * m.Gx + ix] += s;
    }
}

// LDA: Slater exchange + Perdew-Wang correlation (spin-unpolarised).
__global__ void k_lda(long long n, const double *rho, double *vxc, double *exc) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double r = rho[i];
    double e = 0.0, v = 0.0;
    if (r >= 1e-14) {
        const double PI = 3.14159265358979323846;
        const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
        const double r13 = cbrt(r);
        const double rs = cbrt(3.0 / (4.0 * PI)) / r13;
        const double ex = -0.75 * cbrt(3.0 / PI) * r13;
        const double srs = sqrt(rs);
        const double q0 = -2.0 * A * (1.0 + a1 * rs);
        const double q1 = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
        const double dq1 = A * (b1 / srs + 2.0 * b2 + 3.0 * b3 * srs + 4.0 * b4 * rs);
        const double lg = log(1.0 + 1.0 / q1);
        const double ec = q0 * lg;
        const double dec = -2.0 * A * a1 * lg - q0 * dq1 / (q1 * q1 + q1);
        e = ex + ec;
        v = 4.0 / 3.0 * ex + ec - rs / 3.0 * dec;
    }
    if (vxc) vxc[i] = v;
    if (exc) exc[i] = e;
}

// b_sm(x_q) = sum_I -Z_I pi^-3/2 alpha^-3 exp(-|x - R_I|^2 / alpha^2)  (mode 0)
// rho0(x_q) = sum_I Z_I (kappa/pi)^3/2 exp(-kappa |x - R_I|^2)         (mode 1)
__global__ void k_gaussians(MeshDev m, Tables1D T, int natoms, const double *atoms, const double *Z, double width,
                            int mode, double *out) {
    const long long n = (long long)m.nx * m.ny * m.nz * m.nq3;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i / m.nq3), q = (int)(i % m.nq3);
    double x, y, z;
    quad_point(m, T.xq, c, q, x, y, z);
    const double PI = 3.14159265358979323846;
    double s = 0.0;
    for (int I = 0; I < natoms; ++I) {
        const double dx = x - atoms[3 * I], dy = y - atoms[3 * I + 1], dz = z - atoms[3 * I + 2];
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (mode == 0)
            s -= Z[I] * pow(PI, -1.5) / (width * width * width) * exp(-d2 / (width * width));
        else
            s += Z[I] * pow(width / PI, 1.5) * exp(-width * d2);
    }
    out[i] = s;
}

// sum over quadrature points of w_q J a(q) [b(q)] -> block partials
__global__ void k_integrate(MeshDev m, Tables1D T, const double *a, const double *b, double *part) {
    __shared__ double red[32];
    const long long n = (long long)m.nx * m.ny * m.nz * m.nq3;
    const double J = 0.125 * m.h * m.h * m.h;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i % m.nq3);
        const int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        const double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J;
        s += w * a[i] * (b ? b[i] : 1.0);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// Fermi level by bisection on 2 sum f = N_e, then occupations (one block)
__global__ void k_fermi(int N, const double *eig, double ne, double kT, double *out_mu, double *occ) {
    __shared__ double red[32];
    __shared__ double lohi[3];
    __shared__ int done;
    if (threadIdx.x == 0) {
        double mn = eig[0], mx = eig[0];
        for (int i = 1; i < N; ++i) { mn = fmin(mn, eig[i]); mx = fmax(mx, eig[i]); }
        lohi[0] = mn - 50.0 * kT - 1.0;
        lohi[1] = mx + 50.0 * kT + 1.0;
        done = 0;
    }
    __syncthreads();
    for (int it = 0; it < 400; ++it) {
        const double mu = 0.5 * (lohi[0] + lohi[1]);
        double s = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) s += 2.0 * 0.5 * (1.0 - tanh(0.5 * (eig[i] - mu) / kT));
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            lohi[2] = mu;
            if (fabs(t - ne) < 1e-12) done = 1;
            else if (t > ne) lohi[1] = mu;
            else lohi[0] = mu;
        }
        __syncthreads();
        if (done) break;
    }
    const double mu = done ? lohi[2] : 0.5 * (lohi[0] + lohi[1]);
    for (int i = threadIdx.x; i < N; i += blockDim.x) occ[i] = 0.5 * (1.0 - tanh(0.5 * (eig[i] - mu) / kT));
    if (threadIdx.x == 0) *out_mu = mu;
}

__global__ void k_axpy_n(long long n, double a, const double *x, double b, const double *y, double *out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}
__global__ void k_mul_n(long long n, const double *a, const double *b, double *out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * b[i];
}
__global__ void k_add3(long long n, const double *a, const double *b, double *out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}
__global__ void k_scale_n(long long n, double s, double *x) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) x[i] *= s;
}
__global__ void k_dotp(long long n, const double *a, const double *b, double *part) {
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
// weighted dot over quadrature fields (Anderson inner product)
__global__ void k_wdot(MeshDev m, Tables1D T, const double *a, const double *b, double *part) {
    __shared__ double red[32];
    const long long n = (long long)m.nx * m.ny * m.nz * m.nq3;
    const double J = 0.125 * m.h * m.h * m.h;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i % m.nq3);
        const int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        s += T.wq[qx] * T.wq[qy] * T.wq[qz] * J * a[i] * b[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

constexpr int NRED = 512;

}  // namespace

// ===========================================================================
// library-internal helpers
// ===========================================================================
struct ScfState {
    bool ready = false;
    double *d_b = nullptr;          // b_sm at quadrature points
    double *d_avals = nullptr;      // enrichment values per pair and point
    int *d_cell_pair_ptr = nullptr, *d_cell_pair_idx = nullptr, *d_pair_atom = nullptr;
    double *d_Kpois = nullptr;      // (1/4pi) K_e shared cell matrix
    double *d_dinv = nullptr;       // Jacobi preconditioner of the Poisson matrix
    double *d_part = nullptr;       // reduction partials
    double *d_Z = nullptr;          // valence charges
};

static ScfState &scf_state(efe_ctx *ctx) {
    if (!ctx->scf) ctx->scf = new ScfState();
    return *static_cast<ScfState *>(ctx->scf);
}

void efe_scf_free(efe_ctx *ctx) {
    if (!ctx->scf) return;
    ScfState *S = static_cast<ScfState *>(ctx->scf);
    void *ptrs[] = {S->d_b, S->d_avals, S->d_cell_pair_ptr, S->d_cell_pair_idx, S->d_pair_atom, S->d_Kpois,
                    S->d_dinv, S->d_part, S->d_Z};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete S;
    ctx->scf = nullptr;
}


static efe_status reduce_host(efe_ctx *ctx, ScfState &S, double &out) {
    std::vector<double> h(NRED);
    EFE_CUDA(ctx, cudaMemcpyAsync(h.data(), S.d_part, sizeof(double) * NRED, cudaMemcpyDeviceToHost, ctx->stream));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    out = 0.0;
    for (double v : h) out += v;
    return EFE_OK;
}

static efe_status scf_prepare(efe_ctx *ctx) {
    ScfState &S = scf_state(ctx);
    if (S.ready) return EFE_OK;
    const MeshDev &m = ctx->m;
    const long long nq = ctx->n_quad;
    Tables1D T = make_tables(ctx);
    EFE_TRY(efe_alloc(ctx, (void **)&S.d_b, sizeof(double) * nq));
    EFE_TRY(efe_alloc(ctx, (void **)&S.d_part, sizeof(double) * NRED));
    EFE_TRY(efe_alloc(ctx, (void **)&S.d_Z, sizeof(double) * std::max(1, ctx->natoms)));
    if (ctx->natoms)
        EFE_CUDA(ctx, cudaMemcpy(S.d_Z, ctx->zval.data(), sizeof(double) * ctx->natoms, cudaMemcpyHostToDevice));
    k_gaussians<<<nb(nq, 256), 256, 0, ctx->stream>>>(m, T, ctx->natoms, ctx->d_atoms, S.d_Z, ctx->rloc, 0, S.d_b);
    // Poisson cell matrix (1/4pi) K_e = (1/2pi) (1/2 K_e) and its assembled diagonal
    const int ne = m.ne;
    std::vector<double> Kh((size_t)ne * ne);
    EFE_CUDA(ctx, cudaMemcpy(Kh.data(), ctx->d_Khat, sizeof(double) * ne * ne, cudaMemcpyDeviceToHost));
    for (double &v : Kh) v /= (2.0 * kPi);
    EFE_TRY(efe_alloc(ctx, (void **)&S.d_Kpois, sizeof(double) * ne * ne));
    EFE_CUDA(ctx, cudaMemcpy(S.d_Kpois, Kh.data(), sizeof(double) * ne * ne, cudaMemcpyHostToDevice));
    std::vector<double> Kd((size_t)ne * ne, 0.0);
    for (int l = 0; l < ne; ++l) Kd[(size_t)l * ne + l] = Kh[(size_t)l * ne + l];
    double *d_Kd = nullptr, *d_ones = nullptr;
    EFE_TRY(efe_alloc(ctx, (void **)&d_Kd, sizeof(double) * ne * ne));
    EFE_TRY(efe_alloc(ctx, (void **)&d_ones, sizeof(double) * ctx->n_nodes));
    EFE_TRY(efe_alloc(ctx, (void **)&S.d_dinv, sizeof(double) * ctx->n_nodes));
    EFE_CUDA(ctx, cudaMemcpy(d_Kd, Kd.data(), sizeof(double) * ne * ne, cudaMemcpyHostToDevice));
    std::vector<double> ones(ctx->n_nodes, 1.0);
    EFE_CUDA(ctx, cudaMemcpy(d_ones, ones.data(), sizeof(double) * ctx->n_nodes, cudaMemcpyHostToDevice));
    EFE_TRY(efe_cells_shared(ctx, d_Kd, d_ones, S.d_dinv, 1));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<double> dg(ctx->n_nodes);
    EFE_CUDA(ctx, cudaMemcpy(dg.data(), S.d_dinv, sizeof(double) * ctx->n_nodes, cudaMemcpyDeviceToHost));
    for (auto &v : dg) v = (v != 0.0) ? 1.0 / v : 0.0;
    EFE_CUDA(ctx, cudaMemcpy(S.d_dinv, dg.data(), sizeof(double) * ctx->n_nodes, cudaMemcpyHostToDevice));
    cudaFree(d_Kd);
    cudaFree(d_ones);
    // enrichment values at the quadrature points of every pair, and cell -> pairs
    if (ctx->enrich && ctx->natoms) {
        const int np = (int)ctx->pairs.size();
        EFE_TRY(efe_alloc(ctx, (void **)&S.d_avals, sizeof(double) * (size_t)np * 4 * m.nq3));
        FuncParams fp = make_fp(ctx);
        k_pair_values<<<np, 256, 0, ctx->stream>>>(m, T, fp, ctx->d_pairs, ctx->d_atoms, S.d_avals);
        EFE_TRY(efe_check_launch(ctx, "k_pair_values"));
        const int ncell = m.nx * m.ny * m.nz;
        std::vector<int> cnt(ncell + 1, 0), idx(np), atom(np);
        for (int k = 0; k < np; ++k) {
            cnt[ctx->pairs[k].cell + 1]++;
            atom[k] = ctx->pairs[k].atom;
        }
        for (int c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
        std::vector<int> fill(cnt.begin(), cnt.end() - 1);
        for (int k = 0; k < np; ++k) idx[fill[ctx->pairs[k].cell]++] = k;
        EFE_TRY(efe_alloc(ctx, (void **)&S.d_cell_pair_ptr, sizeof(int) * (ncell + 1)));
        EFE_TRY(efe_alloc(ctx, (void **)&S.d_cell_pair_idx, sizeof(int) * std::max(1, np)));
        EFE_TRY(efe_alloc(ctx, (void **)&S.d_pair_atom, sizeof(int) * std::max(1, np)));
        EFE_CUDA(ctx, cudaMemcpy(S.d_cell_pair_ptr, cnt.data(), sizeof(int) * (ncell + 1), cudaMemcpyHostToDevice));
        EFE_CUDA(ctx, cudaMemcpy(S.d_cell_pair_idx, idx.data(), sizeof(int) * np, cudaMemcpyHostToDevice));
        EFE_CUDA(ctx, cudaMemcpy(S.d_pair_atom, atom.data(), sizeof(int) * np, cudaMemcpyHostToDevice));
    }
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    S.ready = true;
    return EFE_OK;
}

static efe_status integrate(efe_ctx *ctx, const double *a, const double *b, double &out) {
    ScfState &S = scf_state(ctx);
    Tables1D T = make_tables(ctx);
    k_integrate<<<NRED, 256, 0, ctx->stream>>>(ctx->m, T, a, b, S.d_part);
    EFE_TRY(efe_check_launch(ctx, "k_integrate"));
    return reduce_host(ctx, S, out);
}

static efe_status dot(efe_ctx *ctx, long long n, const double *a, const double *b, double &out) {
    ScfState &S = scf_state(ctx);
    k_dotp<<<NRED, 256, 0, ctx->stream>>>(n, a, b, S.d_part);
    return reduce_host(ctx, S, out);
}

// values at the quadrature points of FE block U (+ enrichment Ue) -- density or values
static efe_status cell_values(efe_ctx *ctx, const double *U, const double *Ue, int N, const double *w2, int mode,
                              double *out) {
    ScfState &S = scf_state(ctx);
    const MeshDev &m = ctx->m;
    Tables1D T = make_tables(ctx);
    const size_t shm = sizeof(double) * (m.ne * TJ + m.np1 * m.np1 * m.nq + m.np1 * m.nq * m.nq + m.nq * m.np1);
    EFE_CUDA(ctx, cudaFuncSetAttribute(k_cell_values, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const bool enr = ctx->enrich && ctx->natoms && Ue;
    k_cell_values<<<m.nx * m.ny * m.nz, 256, shm, ctx->stream>>>(
        m, T, U, Ue, N, enr ? S.d_cell_pair_ptr : nullptr, S.d_cell_pair_idx, S.d_pair_atom, S.d_avals, w2, mode, out);
    ctx->launches++;
    return efe_check_launch(ctx, "k_cell_values");
}

// FE solution of -1/(4 pi) Lap phi = f, phi = 0 on the box (Jacobi CG)
static efe_status poisson(efe_ctx *ctx, const double *fq, double *phi, double *phi_q, double tol, int max_it,
                          int *iters, double *rel_res) {
    ScfState &S = scf_state(ctx);
    const MeshDev &m = ctx->m;
    const long long n = ctx->n_nodes;
    Tables1D T = make_tables(ctx);
    double *F = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;
    std::vector<void *> own;
    for (double **pp : {&F, &r, &z, &p, &Ap}) {
        EFE_TRY(efe_alloc(ctx, (void **)pp, sizeof(double) * n));
        own.push_back(*pp);
    }
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void *q : own) cudaFree(q);
    };
    EFE_CUDA(ctx, cudaMemsetAsync(F, 0, sizeof(double) * n, ctx->stream));
    const size_t shm = sizeof(double) * (m.nq3 + m.nq * m.nq * m.np1 + m.nq * m.np1 * m.np1);
    EFE_CUDA(ctx, cudaFuncSetAttribute(k_project_colour, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    for (int colour = 0; colour < 8; ++colour) {
        const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
        const int nblocks = ((m.nx - ox + 1) / 2) * ((m.ny - oy + 1) / 2) * ((m.nz - oz + 1) / 2);
        if (nblocks) k_project_colour<<<nblocks, 256, shm, ctx->stream>>>(m, T, colour, fq, F);
    }
    EFE_TRY(efe_check_launch(ctx, "k_project_colour"));
    double bnorm2;
    EFE_TRY(dot(ctx, n, F, F, bnorm2));
    const double bnorm = std::sqrt(bnorm2);
    EFE_CUDA(ctx, cudaMemsetAsync(phi, 0, sizeof(double) * n, ctx->stream));
    int it = 0;
    double rr = bnorm;
    if (bnorm > 0.0) {
        EFE_CUDA(ctx, cudaMemcpyAsync(r, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        k_mul_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, S.d_dinv, r, z);
        EFE_CUDA(ctx, cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        double rz;
        EFE_TRY(dot(ctx, n, r, z, rz));
        while (it < max_it) {
            EFE_TRY(efe_cells_shared(ctx, S.d_Kpois, p, Ap, 1));
            double pAp;
            EFE_TRY(dot(ctx, n, p, Ap, pAp));
            const double alpha = rz / pAp;
            k_axpy_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, 1.0, phi, alpha, p, phi);
            k_axpy_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, 1.0, r, -alpha, Ap, r);
            ++it;
            double r2;
            EFE_TRY(dot(ctx, n, r, r, r2));
            rr = std::sqrt(r2);
            if (rr < tol * bnorm) break;
            k_mul_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, S.d_dinv, r, z);
            double rz_new;
            EFE_TRY(dot(ctx, n, r, z, rz_new));
            k_axpy_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, 1.0, z, rz_new / rz, p, p);
            rz = rz_new;
        }
    }
    if (phi_q) EFE_TRY(cell_values(ctx, phi, nullptr, 1, nullptr, 1, phi_q));
    cleanup();
    if (iters) *iters = it;
    if (rel_res) *rel_res = bnorm > 0 ? rr / bnorm : 0.0;
    return EFE_OK;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

efe_status efe_smeared_charge(efe_ctx *ctx, double *b_q) {
    if (!ctx || !b_q) return EFE_ERR_ARG;
    EFE_TRY(scf_prepare(ctx));
    EFE_CUDA(ctx, cudaMemcpyAsync(b_q, scf_state(ctx).d_b, sizeof(double) * ctx->n_quad, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

efe_status efe_atomic_density(efe_ctx *ctx, double kappa, double *rho_q) {
    if (!ctx || !rho_q || !(kappa > 0)) return EFE_ERR_ARG;
    EFE_TRY(scf_prepare(ctx));
    Tables1D T = make_tables(ctx);
    k_gaussians<<<nb(ctx->n_quad, 256), 256, 0, ctx->stream>>>(ctx->m, T, ctx->natoms, ctx->d_atoms,
                                                                scf_state(ctx).d_Z, kappa, 1, rho_q);
    EFE_TRY(efe_check_launch(ctx, "k_gaussians"));
    double tot;
    EFE_TRY(integrate(ctx, rho_q, nullptr, tot));
    double ne = 0.0;
    for (double z : ctx->zval) ne += z;
    if (tot > 0) k_scale_n<<<nb(ctx->n_quad, 256), 256, 0, ctx->stream>>>(ctx->n_quad, ne / tot, rho_q);
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

efe_status efe_density(efe_ctx *ctx, const double *X, int N, const double *occ, double *rho_q) {
    if (!ctx || !X || !occ || !rho_q || N <= 0) return EFE_ERR_ARG;
    EFE_TRY(scf_prepare(ctx));
    const long long nn = ctx->n_nodes;
    double *Xp = nullptr, *w2 = nullptr;
    EFE_TRY(efe_alloc(ctx, (void **)&Xp, sizeof(double) * (size_t)nn * N));
    EFE_TRY(efe_alloc(ctx, (void **)&w2, sizeof(double) * N));
    std::vector<double> h(N);
    for (int j = 0; j < N; ++j) h[j] = 2.0 * occ[j];
    EFE_CUDA(ctx, cudaMemcpyAsync(w2, h.data(), sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
    efe_status st = efe_xprime_fp64(ctx, X, Xp, N);
    if (st == EFE_OK) st = cell_values(ctx, Xp, X + nn * N, N, w2, 0, rho_q);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(Xp);
    cudaFree(w2);
    return st;
}

efe_status efe_xc(efe_ctx *ctx, const double *rho_q, double *vxc_q, double *exc_q) {
    if (!ctx || !rho_q) return EFE_ERR_ARG;
    k_lda<<<nb(ctx->n_quad, 256), 256, 0, ctx->stream>>>(ctx->n_quad, rho_q, vxc_q, exc_q);
    EFE_TRY(efe_check_launch(ctx, "k_lda"));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

efe_status efe_poisson(efe_ctx *ctx, const double *f_q, double *phi_nodes, double *phi_q, double tol, int max_it,
                       int *iters, double *rel_res) {
    if (!ctx || !f_q || !phi_nodes || !(tol > 0) || max_it < 1) return EFE_ERR_ARG;
    EFE_TRY(scf_prepare(ctx));
    EFE_TRY(poisson(ctx, f_q, phi_nodes, phi_q, tol, max_it, iters, rel_res));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}

efe_status efe_fermi(efe_ctx *ctx, const double *eig, int N, double n_elec, double kT, double *mu, double *occ) {
    if (!ctx || !eig || !mu || !occ || N <= 0 || !(kT > 0)) return EFE_ERR_ARG;
    double *d = nullptr;
    EFE_TRY(efe_alloc(ctx, (void **)&d, sizeof(double) * (2 * N + 1)));
    EFE_CUDA(ctx, cudaMemcpyAsync(d, eig, sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream));
    k_fermi<<<1, 256, 0, ctx->stream>>>(N, d, n_elec, kT, d + 2 * N, d + N);
    efe_status st = efe_check_launch(ctx, "k_fermi");
    if (st == EFE_OK) {
        if (cudaMemcpyAsync(occ, d + N, sizeof(double) * N, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaMemcpyAsync(mu, d + 2 * N, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            st = EFE_ERR_CUDA;
    }
    cudaStreamSynchronize(ctx->stream);
    cudaFree(d);
    return st;
}

efe_status efe_integrate(efe_ctx *ctx, const double *a_q, const double *b_q, double *out) {
    if (!ctx || !a_q || !out) return EFE_ERR_ARG;
    EFE_TRY(scf_prepare(ctx));
    return integrate(ctx, a_q, b_q, *out);
}

efe_status efe_scf(efe_ctx *ctx, const efe_scf_opts *o, double *X, int N, const double *u0, const double *rho0_q,
                   efe_scf_result *res) {
    if (!ctx || !o || !X || !u0 || !res || N <= 0 || o->cheb_degree < 2 || o->max_iter < 1) return EFE_ERR_ARG;
    EFE_TRY(scf_prepare(ctx));
    ScfState &S = scf_state(ctx);
    const long long nq = ctx->n_quad, nn = ctx->n_nodes, rows = ctx->n_rows;
    const int hist = std::max(0, o->mix_history);
    double ne = 0.0;
    for (double z : ctx->zval) ne += z;
    const double kT = 3.166811563e-6 * o->temperature;
    const int nocc = (int)std::ceil(ne / 2.0);
    const double alpha = ctx->rloc;
    // closed-form electrostatic constants (Gaussian smeared charges)
    double eself = 0.0, dzz = 0.0;
    for (int I = 0; I < ctx->natoms; ++I) {
        eself += ctx->zval[I] * ctx->zval[I] / (std::sqrt(2.0 * kPi) * alpha);
        for (int J = I + 1; J < ctx->natoms; ++J) {
            double dx = ctx->xyz[3 * I] - ctx->xyz[3 * J], dy = ctx->xyz[3 * I + 1] - ctx->xyz[3 * J + 1],
                   dz = ctx->xyz[3 * I + 2] - ctx->xyz[3 * J + 2];
            double R = std::sqrt(dx * dx + dy * dy + dz * dz);
            dzz += ctx->zval[I] * ctx->zval[J] * std::erfc(R / (std::sqrt(2.0) * alpha)) / R;
        }
    }
    // buffers
    std::vector<void *> own;
    auto take = [&](size_t bytes) -> double * {
        void *p = nullptr;
        if (efe_alloc(ctx, &p, bytes) != EFE_OK) return nullptr;
        own.push_back(p);
        return (double *)p;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void *p : own) cudaFree(p);
    };
    const int HS = hist + 1;
    double *rho_in = take(sizeof(double) * nq), *rho_out = take(sizeof(double) * nq), *veff = take(sizeof(double) * nq),
           *vxc = take(sizeof(double) * nq), *exc = take(sizeof(double) * nq), *phi = take(sizeof(double) * nn),
           *phi_q = take(sizeof(double) * nq), *tmp = take(sizeof(double) * nq),
           *HX = take(sizeof(double) * rows * N), *Vout = take(sizeof(double) * rows * N),
           *dlam = take(sizeof(double) * N), *hin = take(sizeof(double) * nq * HS), *hout = take(sizeof(double) * nq * HS);
    if (!rho_in || !rho_out || !veff || !vxc || !exc || !phi || !phi_q || !tmp || !HX || !Vout || !dlam || !hin ||
        !hout) {
        cleanup();
        return EFE_ERR_OOM;
    }
    efe_status st = EFE_OK;
#define SCF_TRY(x)                 \
    do {                           \
        if ((st = (x)) != EFE_OK) { \
            cleanup();             \
            return st;             \
        }                          \
    } while (0)
    if (rho0_q) {
        if (cudaMemcpyAsync(rho_in, rho0_q, sizeof(double) * nq, cudaMemcpyDeviceToDevice, ctx->stream) != cudaSuccess) {
            cleanup();
            return EFE_ERR_CUDA;
        }
    } else {
        SCF_TRY(efe_atomic_density(ctx, o->kappa > 0 ? o->kappa : 2.4, rho_in));
    }
    Tables1D T = make_tables(ctx);
    std::vector<double> eig(N), resid(N), occ(N), lam(N);
    double E = 0.0, F = 0.0, mu = 0.0, E_prev = 0.0, dr = 0.0, dE = 0.0;
    bool have_prev = false, conv = false;
    int nh = 0;                       // history entries stored (ring of HS)
    int it = 0;
    const efe_precision prec = (efe_precision)o->precision;
    res->poisson_iters = 0;
    for (it = 1; it <= o->max_iter; ++it) {
        int pit = 0;
        // v_eff = v_xc[rho_in] + phi[rho_in + b]
        k_add3<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_in, S.d_b, tmp);
        SCF_TRY(poisson(ctx, tmp, phi, phi_q, o->poisson_tol, 100000, &pit, nullptr));
        res->poisson_iters += pit;
        k_lda<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_in, vxc, nullptr);
        k_add3<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, vxc, phi_q, veff);
        SCF_TRY(efe_potential_assembly(ctx, veff));
        if (it == 1) {
            int passes = 0;
            st = efe_chfsi(ctx, X, HX, N, o->cheb_degree, nullptr, u0, o->first_max_pass, o->first_tol, nocc, prec,
                           eig.data(), resid.data(), &passes);
            if (st != EFE_OK && st != EFE_ERR_NO_CONVERGE) {
                cleanup();
                return st;
            }
        } else {
            double lz[3];
            SCF_TRY(efe_lanczos(ctx, u0, 10, lz));
            SCF_TRY(efe_apply_h(ctx, X, HX, N, EFE_FP64));
            if (cudaMemcpyAsync(dlam, eig.data(), sizeof(double) * N, cudaMemcpyHostToDevice, ctx->stream) !=
                cudaSuccess) {
                cleanup();
                return EFE_ERR_CUDA;
            }
            const double bd[3] = {eig[0], eig[N - 1], lz[2]};
            SCF_TRY(efe_filter(ctx, X, HX, dlam, N, o->cheb_degree, bd, prec, Vout));
            SCF_TRY(efe_rayleigh_ritz(ctx, Vout, HX, N, eig.data(), resid.data()));
            if (cudaMemcpyAsync(X, Vout, sizeof(double) * rows * N, cudaMemcpyDeviceToDevice, ctx->stream) !=
                cudaSuccess) {
                cleanup();
                return EFE_ERR_CUDA;
            }
        }
        SCF_TRY(efe_fermi(ctx, eig.data(), N, ne, kT, &mu, occ.data()));
        SCF_TRY(efe_density(ctx, X, N, occ.data(), rho_out));
        if (o->renormalize) {
            double tot;
            SCF_TRY(integrate(ctx, rho_out, nullptr, tot));
            k_scale_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, ne / tot, rho_out);
        }
        // energies
        k_add3<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_out, S.d_b, tmp);
        SCF_TRY(poisson(ctx, tmp, phi, phi_q, o->poisson_tol, 100000, &pit, nullptr));
        res->poisson_iters += pit;
        k_lda<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_out, nullptr, exc);
        double i_rv, i_rexc, i_hart;
        SCF_TRY(integrate(ctx, rho_out, veff, i_rv));
        SCF_TRY(integrate(ctx, rho_out, exc, i_rexc));
        SCF_TRY(integrate(ctx, tmp, phi_q, i_hart));
        double band = 0.0, ent = 0.0;
        for (int j = 0; j < N; ++j) {
            band += 2.0 * occ[j] * eig[j];
            const double f = std::min(1.0, std::max(0.0, occ[j]));
            if (f > 0.0 && f < 1.0) ent += f * std::log(f) + (1.0 - f) * std::log(1.0 - f);
        }
        E = band - i_rv + i_rexc + 0.5 * i_hart - eself + dzz;
        F = E + 2.0 * kT * ent;
        k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_out, -1.0, rho_in, tmp);
        double d2;
        SCF_TRY(integrate(ctx, tmp, tmp, d2));
        dr = std::sqrt(std::max(d2, 0.0)) / ne;
        dE = have_prev ? std::fabs(E - E_prev) / std::max(1, ctx->natoms) : 1e300;
        if (o->log) o->log(o->log_user, it, E, F, mu, dr, dE, resid[0]);
        if (dr < o->tol_rho && dE < o->tol_e) {
            conv = true;
            break;
        }
        E_prev = E;
        have_prev = true;
        // Anderson (Walker-Ni form) on the quadrature-point densities
        const int slot = nh % HS;
        cudaMemcpyAsync(hin + (size_t)slot * nq, rho_in, sizeof(double) * nq, cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemcpyAsync(hout + (size_t)slot * nq, rho_out, sizeof(double) * nq, cudaMemcpyDeviceToDevice, ctx->stream);
        ++nh;
        const int have = std::min(nh, HS);           // entries, oldest first
        auto at = [&](double *base, int k) { return base + (size_t)((nh - have + k) % HS) * nq; };
        const int mm = have - 1;
        double *xk = at(hin, mm);
        // R_k = out_k - in_k (into tmp)
        k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, at(hout, mm), -1.0, xk, tmp);
        std::vector<double> gamma(mm, 0.0);
        if (mm > 0) {
            // dR_j = R_{j+1} - R_j ; A = dR^T W dR, b = dR^T W R_k (normal equations)
            double *dRj = nullptr, *dRi = nullptr;
            dRj = take(sizeof(double) * nq);
            dRi = take(sizeof(double) * nq);
            if (!dRj || !dRi) { cleanup(); return EFE_ERR_OOM; }
            std::vector<double> A(mm * mm), bvec(mm);
            auto make_dR = [&](int j, double *out) {
                // (out_{j+1} - in_{j+1}) - (out_j - in_j)
                k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, at(hout, j + 1), -1.0, at(hin, j + 1), out);
                k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, out, -1.0, at(hout, j), out);
                k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, out, 1.0, at(hin, j), out);
            };
            for (int i = 0; i < mm; ++i) {
                make_dR(i, dRi);
                for (int j = i; j < mm; ++j) {
                    make_dR(j, dRj);
                    double v;
                    k_wdot<<<NRED, 256, 0, ctx->stream>>>(ctx->m, T, dRi, dRj, S.d_part);
                    SCF_TRY(reduce_host(ctx, S, v));
                    A[i * mm + j] = A[j * mm + i] = v;
                }
                double v;
                k_wdot<<<NRED, 256, 0, ctx->stream>>>(ctx->m, T, dRi, tmp, S.d_part);
                SCF_TRY(reduce_host(ctx, S, v));
                bvec[i] = v;
            }
            // least squares by the pseudo-inverse (eigen-decomposition of A)
            std::vector<double> w, Vv;
            efe_sym_eig(mm, A, w, Vv);
            double wmax = 0.0;
            for (double x : w) wmax = std::max(wmax, std::fabs(x));
            const double cut = wmax * 2.220446049250313e-16 * mm;
            for (int k = 0; k < mm; ++k) {
                if (std::fabs(w[k]) <= cut) continue;
                double proj = 0.0;
                for (int i = 0; i < mm; ++i) proj += Vv[i * mm + k] * bvec[i];
                for (int i = 0; i < mm; ++i) gamma[i] += Vv[i * mm + k] * proj / w[k];
            }
            cudaStreamSynchronize(ctx->stream);
            cudaFree(dRj);
            cudaFree(dRi);
            own.pop_back();
            own.pop_back();
        }
        // rho_next = (x_k - dX gamma) + beta (R_k - dR gamma), built in rho_in
        k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, xk, o->mix_beta, tmp, rho_in);
        for (int j = 0; j < mm; ++j) {
            if (gamma[j] == 0.0) continue;
            // dX_j = in_{j+1} - in_j ; dR_j = (out_{j+1}-in_{j+1}) - (out_j-in_j)
            const double gj = gamma[j], bt = o->mix_beta;
            // rho -= g (in_{j+1} - in_j) + beta g (dR_j)
            k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_in, -gj * (1.0 - bt), at(hin, j + 1), rho_in);
            k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_in, gj * (1.0 - bt), at(hin, j), rho_in);
            k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_in, -gj * bt, at(hout, j + 1), rho_in);
            k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_in, gj * bt, at(hout, j), rho_in);
        }
        if (cudaGetLastError() != cudaSuccess) {
            cleanup();
            return EFE_ERR_CUDA;
        }
    }
#undef SCF_TRY
    res->E = E;
    res->F = F;
    res->mu = mu;
    res->iters = std::min(it, o->max_iter);
    res->converged = conv ? 1 : 0;
    res->drho = dr;
    res->dE = dE;
    if (res->eig) std::copy(eig.begin(), eig.end(), res->eig);
    if (res->rho_q) cudaMemcpyAsync(res->rho_q, rho_out, sizeof(double) * nq, cudaMemcpyDeviceToDevice, ctx->stream);
    cleanup();
    return conv ? EFE_OK : EFE_ERR_NO_CONVERGE;
}

}  // extern "C"
