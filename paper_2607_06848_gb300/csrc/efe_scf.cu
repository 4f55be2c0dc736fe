// Self-consistent field machinery on the GPU (paper Sec. II.A, Sec. IV):
// density at the quadrature points (Eq. rhocompute), Fermi level (Eq.
// electronconstraint) at 500 K, LDA exchange-correlation in the Perdew-Wang
// form, the electrostatic potential of rho + b_sm by FE conjugate gradients
// (Eqs. EellocReform, poisson), energies, Anderson mixing, and the SCF loop.
#include "efe_internal.cuh"
#include "efe_funcs.cuh"

#include <algorithm>
#include <chrono>
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
// Y += s M^cc X (lumped mass, zero on the Dirichlet rows)
__global__ void k_add_mass(long long n, double s, const double *mcc, const double *X, double *Y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) Y[i] += s * mcc[i] * X[i];
}
// Jacobi of (1/4pi) K + s M^cc from that of (1/4pi) K (rows with dinv = 0 stay 0)
__global__ void k_shift_jacobi(long long n, double s, const double *mcc, const double *dinv, double *out) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) out[i] = dinv[i] != 0.0 ? 1.0 / (1.0 / dinv[i] + s * mcc[i]) : 0.0;
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
constexpr int NRED = 512;

// --- the Poisson operator by sum factorisation -------------------------------
// On a cube cell with Gauss quadrature the stiffness integrand separates, so
// (1/4 pi) K_e = c (S x M x M + M x S x M + M x M x S) with the 1-D matrices
// S_ab = sum_q w_q N'_a N'_b, M_ab = sum_q w_q N_a N_b on [-1, 1] and
// c = (h/2) / (4 pi).  Applied as w1 = M_z u, w2 = S_z u; t1 = M_y w1,
// t2 = S_y w1 + M_y w2; y = S_x t1 + M_x t2: 7 (p+1)^4 FMAs per cell instead
// of (p+1)^6 for the dense matrix.  One CTA per cell of one colour.
template <typename T>
struct Lap1 {
    T S[(EFE_MAXP + 1) * (EFE_MAXP + 1)], M[(EFE_MAXP + 1) * (EFE_MAXP + 1)];
    T c;
};
using Lap1D = Lap1<double>;

// T = double: the operator of the FP64 CG; T = float: of the inner FP32 CG of
// the mixed-precision solve (the correction equation; its residual is formed
// in FP64 by the double instance)
constexpr int kLapMax = (EFE_MAXP + 1) * (EFE_MAXP + 1) * (EFE_MAXP + 1);
template <typename T>
__global__ void __launch_bounds__(256) k_lap_colour(MeshDev m, Lap1<T> L, int colour, const T *X, T *Y) {
    __shared__ T u[kLapMax], w1[kLapMax], w2[kLapMax], w3[kLapMax];
    const int np1 = m.np1, ne = m.ne;
    const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
    const int hx = (m.nx - ox + 1) / 2, hy = (m.ny - oy + 1) / 2;
    const int b = blockIdx.x;
    const int cx = 2 * (b % hx) + ox, cy = 2 * ((b / hx) % hy) + oy, cz = 2 * (b / (hx * hy)) + oz;
    for (int l = threadIdx.x; l < ne; l += blockDim.x) {
        const int ax = l % np1, ay = (l / np1) % np1, az = l / (np1 * np1);
        u[l] = X[((long long)(cz * m.p + az) * m.Gy + (cy * m.p + ay)) * m.Gx + (cx * m.p + ax)];
    }
    __syncthreads();
    for (int l = threadIdx.x; l < ne; l += blockDim.x) {         // along z: w1 = M u, w2 = S u
        const int axy = l % (np1 * np1), az = l / (np1 * np1);
        T a = 0, s = 0;
        for (int k = 0; k < np1; ++k) {
            const T v = u[k * np1 * np1 + axy];
            a += L.M[az * np1 + k] * v;
            s += L.S[az * np1 + k] * v;
        }
        w1[l] = a;
        w2[l] = s;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < ne; l += blockDim.x) {         // along y: u = M w1, w3 = S w1 + M w2
        const int ax = l % np1, ay = (l / np1) % np1, az = l / (np1 * np1);
        T a = 0, s = 0;
        for (int k = 0; k < np1; ++k) {
            const int src = (az * np1 + k) * np1 + ax;
            a += L.M[ay * np1 + k] * w1[src];
            s += L.S[ay * np1 + k] * w1[src] + L.M[ay * np1 + k] * w2[src];
        }
        u[l] = a;
        w3[l] = s;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < ne; l += blockDim.x) {         // along x: S u + M w3, scatter
        const int ax = l % np1, ay = (l / np1) % np1, az = l / (np1 * np1);
        const int ix = cx * m.p + ax, iy = cy * m.p + ay, iz = cz * m.p + az;
        if (!interior_node(m, ix, iy, iz)) continue;
        T s = 0;
        for (int k = 0; k < np1; ++k) {
            const int src = (az * np1 + ay) * np1 + k;
            s += L.S[ax * np1 + k] * u[src] + L.M[ax * np1 + k] * w3[src];
        }
        Y[((long long)iz * m.Gy + iy) * m.Gx + ix] += L.c * s;
    }
}

// --- conjugate gradients with the scalars kept on the device ------------------
// sc[]: rz, alpha, beta, threshold tol*||F||, done flag, iterations, ||r||
enum { CG_RZ = 0, CG_ALPHA, CG_BETA, CG_THR, CG_DONE, CG_IT, CG_RR, CG_NSC };

// fixed-order sum of NRED partials by one warp (lane l takes l, l+32, ...)
__device__ __forceinline__ double warp_sum_parts(const double *part) {
    double s = 0.0;
    for (int i = threadIdx.x; i < NRED; i += 32) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    return s;
}

// alpha = rz / (p . Ap), zero once converged
__global__ void k_cg_alpha(const double *part, double *sc) {
    const double pAp = warp_sum_parts(part);
    if (threadIdx.x == 0) sc[CG_ALPHA] = sc[CG_DONE] != 0.0 ? 0.0 : sc[CG_RZ] / pAp;
}

// phi += alpha p; r -= alpha Ap; z = D^-1 r; partials of r.r (part[b]) and r.z (part[NRED + b])
__global__ void k_cg_update(long long n, const double *sc, double *phi, double *r, const double *p,
                            const double *Ap, const double *dinv, double *z, double *part) {
    __shared__ double red[2][32];
    const double a = sc[CG_ALPHA];
    double s1 = 0.0, s2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double ri = r[i];
        if (a != 0.0) {     // alpha = 0 (the start, or after convergence) leaves phi and r as they are
            phi[i] += a * p[i];
            ri -= a * Ap[i];
            r[i] = ri;
        }
        const double zi = dinv[i] * ri;
        z[i] = zi;
        s1 += ri * ri;
        s2 += ri * zi;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        part[blockIdx.x] = t1;
        part[NRED + blockIdx.x] = t2;
    }
}

// convergence test on ||r||, then beta = rz_new / rz (first = true: the start,
// which only records rz and the test)
__global__ void k_cg_beta(const double *part, double *sc, int first) {
    const double r2 = warp_sum_parts(part);
    const double rzn = warp_sum_parts(part + NRED);
    if (threadIdx.x != 0) return;
    if (first) {
        sc[CG_RR] = sqrt(r2);
        sc[CG_RZ] = rzn;
        sc[CG_DONE] = sqrt(r2) < sc[CG_THR] ? 1.0 : 0.0;
        sc[CG_IT] = 0.0;
        return;
    }
    if (sc[CG_DONE] != 0.0) {
        sc[CG_BETA] = 0.0;
        return;
    }
    sc[CG_IT] += 1.0;
    sc[CG_RR] = sqrt(r2);
    if (sqrt(r2) < sc[CG_THR]) {
        sc[CG_DONE] = 1.0;
        sc[CG_BETA] = 0.0;
    } else {
        sc[CG_BETA] = rzn / sc[CG_RZ];
        sc[CG_RZ] = rzn;
    }
}

// p = z + beta p
__global__ void k_cg_p(long long n, const double *sc, const double *z, double *p) {
    const double b = sc[CG_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + b * p[i];
}

__global__ void k_set_scalar(double *sc, int k, double v) { sc[k] = v; }

// --- the FP32 inner CG of the mixed-precision solve --------------------------
// Vectors in FP32, each thread's partial sums in FP32 (a few tens of terms),
// the block and grid sums and the CG scalars in FP64.
__device__ __forceinline__ void block_parts2(double s1, double s2, double *part, int nparts) {
    __shared__ double red[2][32];
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        part[blockIdx.x] = t1;
        if (nparts > 1) part[NRED + blockIdx.x] = t2;
    }
}
__global__ void k_dotp_f(long long n, const float *a, const float *b, double *part) {
    float s = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s = fmaf(a[i], b[i], s);
    block_parts2((double)s, 0.0, part, 1);
}
// d += alpha p; r -= alpha Ap; z = D^-1 r; partials of r.r and r.z
__global__ void k_cg_update_f(long long n, const double *sc, float *d, float *r, const float *p, const float *Ap,
                              const float *dinv, float *z, double *part) {
    const float a = (float)sc[CG_ALPHA];
    float s1 = 0.f, s2 = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float ri = r[i];
        if (a != 0.f) {
            d[i] = fmaf(a, p[i], d[i]);
            ri = fmaf(-a, Ap[i], ri);
            r[i] = ri;
        }
        const float zi = dinv[i] * ri;
        z[i] = zi;
        s1 = fmaf(ri, ri, s1);
        s2 = fmaf(ri, zi, s2);
    }
    block_parts2((double)s1, (double)s2, part, 2);
}
__global__ void k_cg_p_f(long long n, const double *sc, const float *z, float *p) {
    const float b = (float)sc[CG_BETA];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = fmaf(b, p[i], z[i]);
}
__global__ void k_narrow(long long n, const double *x, float *y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}
// phi += d (the correction), and d = 0 for the next inner solve
__global__ void k_add_correction(long long n, double *phi, float *d) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) {
        phi[i] += (double)d[i];
        d[i] = 0.f;
    }
}
__global__ void k_add_mass_f(long long n, float s, const float *mcc, const float *X, float *Y) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) Y[i] = fmaf(s * mcc[i], X[i], Y[i]);
}

// --- Anderson mixing: history rings of rho_in (x) and residuals R = rho_out - rho_in
constexpr int kMixMax = 8;                                           // dR vectors at most
constexpr int kMixNV = kMixMax * (kMixMax + 1) / 2 + kMixMax;       // A (upper) and b
struct MixRing {
    const double *x[kMixMax + 1];    // oldest first
    const double *R[kMixMax + 1];
};
__host__ __device__ constexpr int mix_idx(int i, int j) { return i * kMixMax - i * (i - 1) / 2 + (j - i); }

// partials of A_ij = <dR_i, dR_j>_w (i <= j < mm) and b_i = <dR_i, R_mm>_w,
// dR_j = R_{j+1} - R_j, w the quadrature weights; part[block][kMixNV]
__global__ void __launch_bounds__(256) k_mix_gram(MeshDev m, Tables1D T, MixRing ring, int mm, double *part) {
    __shared__ double red[8][kMixNV];
    const long long n = (long long)m.nx * m.ny * m.nz * m.nq3;
    const double J = 0.125 * m.h * m.h * m.h;
    const double *Rk = ring.R[0];
#pragma unroll
    for (int j = 1; j <= kMixMax; ++j)
        if (j == mm) Rk = ring.R[j];
    double acc[kMixNV];
#pragma unroll
    for (int k = 0; k < kMixNV; ++k) acc[k] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i % m.nq3);
        const int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        const double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J;
        double d[kMixMax];
        double prev = ring.R[0][i];
#pragma unroll
        for (int j = 0; j < kMixMax; ++j) {
            double nxt = 0.0;
            if (j < mm) nxt = ring.R[j + 1][i];
            d[j] = (j < mm) ? nxt - prev : 0.0;
            prev = nxt;
        }
        const double rk = Rk[i];
#pragma unroll
        for (int a = 0; a < kMixMax; ++a) {
            const double wa = w * d[a];
#pragma unroll
            for (int b = a; b < kMixMax; ++b) acc[mix_idx(a, b)] += wa * d[b];
            acc[kMixNV - kMixMax + a] += wa * rk;
        }
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kMixNV; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kMixNV) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
        part[(size_t)blockIdx.x * kMixNV + threadIdx.x] = t;
    }
}

// out[k] = sum over blocks of part[block][k] (fixed order)
__global__ void k_mix_sum(int nblk, const double *part, double *out) {
    const int k = threadIdx.x;
    if (k >= kMixNV) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += part[(size_t)b * kMixNV + k];
    out[k] = t;
}

struct MixCoef {
    double g[kMixMax];
};

// rho = x_mm + beta R_mm - sum_j gamma_j ((x_{j+1} - x_j) + beta (R_{j+1} - R_j))
// rho = xbar + beta Rbar; Rbar also written when Rbar_out is given (preconditioned update)
__global__ void k_mix_update(long long n, MixRing ring, int mm, MixCoef gc, double beta, double *rho,
                             double *Rbar_out) {
    const double *xk = ring.x[0], *Rk = ring.R[0];
#pragma unroll
    for (int j = 1; j <= kMixMax; ++j)
        if (j == mm) {
            xk = ring.x[j];
            Rk = ring.R[j];
        }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double xb = xk[i], rb = Rk[i];
#pragma unroll
        for (int j = 0; j < kMixMax; ++j)
            if (j < mm) {
                xb -= gc.g[j] * (ring.x[j + 1][i] - ring.x[j][i]);
                rb -= gc.g[j] * (ring.R[j + 1][i] - ring.R[j][i]);
            }
        rho[i] = xb + beta * rb;
        if (Rbar_out) Rbar_out[i] = rb;
    }
}

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
    double *d_dinv_shift = nullptr; // the same for (1/4pi)(K + k^2 M^cc), at shift_k2
    double shift_k2 = 0.0;
    double *d_part = nullptr;       // reduction partials
    double *d_Z = nullptr;          // valence charges
    // conjugate-gradient work vectors (n_nodes), scalars and partials
    double *cg_F = nullptr, *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_Ap = nullptr;
    double *cg_sc = nullptr, *cg_part = nullptr;
    Lap1D lap{};                    // 1-D factors of the Poisson operator
    Lap1<float> lapf{};             // the same in FP32 (inner solves)
    // FP32 work vectors of the mixed-precision solve, the FP32 mass, and the
    // FP32 Jacobi factors with the shift they were made for (-1: none yet)
    float *f_r = nullptr, *f_z = nullptr, *f_p = nullptr, *f_Ap = nullptr, *f_d = nullptr, *f_dinv = nullptr,
          *f_mcc = nullptr;
    double f_dinv_k2 = -1.0;
};

static ScfState &scf_state(efe_ctx *ctx) {
    if (!ctx->scf) ctx->scf = new ScfState();
    return *static_cast<ScfState *>(ctx->scf);
}

void efe_scf_free(efe_ctx *ctx) {
    if (!ctx->scf) return;
    ScfState *S = static_cast<ScfState *>(ctx->scf);
    void *ptrs[] = {S->d_b, S->d_avals, S->d_cell_pair_ptr, S->d_cell_pair_idx, S->d_pair_atom, S->d_Kpois,
                    S->d_dinv, S->d_dinv_shift, S->d_part, S->d_Z, S->cg_F, S->cg_r, S->cg_z, S->cg_p, S->cg_Ap, S->cg_sc,
                    S->cg_part, S->f_r, S->f_z, S->f_p, S->f_Ap, S->f_d, S->f_dinv, S->f_mcc};
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
    // 1-D factors of the Poisson operator (Gauss quadrature on [-1, 1])
    {
        const int np1 = m.np1, nq = m.nq;
        for (int a = 0; a < np1; ++a)
            for (int b = 0; b < np1; ++b) {
                double sv = 0.0, mv = 0.0;
                for (int q = 0; q < nq; ++q) {
                    sv += ctx->wq[q] * ctx->D1[q * np1 + a] * ctx->D1[q * np1 + b];
                    mv += ctx->wq[q] * ctx->B1[q * np1 + a] * ctx->B1[q * np1 + b];
                }
                S.lap.S[a * np1 + b] = sv;
                S.lap.M[a * np1 + b] = mv;
            }
        S.lap.c = 0.5 * m.h / (4.0 * kPi);
        for (int i = 0; i < np1 * np1; ++i) {
            S.lapf.S[i] = (float)S.lap.S[i];
            S.lapf.M[i] = (float)S.lap.M[i];
        }
        S.lapf.c = (float)S.lap.c;
    }
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

// Y = (1/4 pi) K X + shift M^cc X for one nodal vector (Dirichlet rows left at zero)
static efe_status lap_apply(efe_ctx *ctx, const double *X, double *Y, double shift = 0.0) {
    ScfState &S = scf_state(ctx);
    const MeshDev &m = ctx->m;
    EFE_CUDA(ctx, cudaMemsetAsync(Y, 0, sizeof(double) * ctx->n_nodes, ctx->stream));
    for (int colour = 0; colour < 8; ++colour) {
        const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
        const int ncol = ((m.nx - ox + 1) / 2) * ((m.ny - oy + 1) / 2) * ((m.nz - oz + 1) / 2);
        if (ncol) k_lap_colour<<<ncol, 256, 0, ctx->stream>>>(m, S.lap, colour, X, Y);
    }
    if (shift != 0.0)
        k_add_mass<<<nb(ctx->n_nodes, 256), 256, 0, ctx->stream>>>(ctx->n_nodes, shift, ctx->d_mcc, X, Y);
    return efe_check_launch(ctx, "k_lap_colour");
}

// the FP32 operator: Y = (1/4 pi) K X + shift M^cc X
static efe_status lap_apply_f(efe_ctx *ctx, const float *X, float *Y, float shift) {
    ScfState &S = scf_state(ctx);
    const MeshDev &m = ctx->m;
    EFE_CUDA(ctx, cudaMemsetAsync(Y, 0, sizeof(float) * ctx->n_nodes, ctx->stream));
    for (int colour = 0; colour < 8; ++colour) {
        const int ox = colour & 1, oy = (colour >> 1) & 1, oz = (colour >> 2) & 1;
        const int ncol = ((m.nx - ox + 1) / 2) * ((m.ny - oy + 1) / 2) * ((m.nz - oz + 1) / 2);
        if (ncol) k_lap_colour<float><<<ncol, 256, 0, ctx->stream>>>(m, S.lapf, colour, X, Y);
    }
    if (shift != 0.f)
        k_add_mass_f<<<nb(ctx->n_nodes, 256), 256, 0, ctx->stream>>>(ctx->n_nodes, shift, S.f_mcc, X, Y);
    return efe_check_launch(ctx, "k_lap_colour<float>");
}

constexpr int kCgBlock = 16;            // CG iterations between host reads of the convergence flag
constexpr double kInnerEta = 1e-4;      // an inner FP32 solve reduces its residual by this factor
constexpr int kMaxOuter = 30;

// Mixed-precision stage of the solve (iterative refinement): the residual
// r = F - A phi in FP64; the correction equation A d = r by Jacobi CG in FP32
// (vectors and per-thread sums in FP32, CG scalars in FP64) to kInnerEta of
// |r|; phi += d in FP64; repeat until |r| < thr.  The FP32 operator does the
// bulk of the iterations on this part's FP32 pipe; the stopping test is on the
// FP64 residual, so the result meets the same tolerance as the FP64 CG.  The
// FP64 residual of the final phi is left in S.cg_r.
static efe_status poisson_mixed(efe_ctx *ctx, ScfState &S, const double *F, double *phi, bool warm, double shift,
                                const double *dinv, double k2, double thr, int max_it, int *iters) {
    const long long n = ctx->n_nodes;
    if (!S.f_r) {
        for (float **pp : {&S.f_r, &S.f_z, &S.f_p, &S.f_Ap, &S.f_d, &S.f_dinv, &S.f_mcc})
            EFE_TRY(efe_alloc(ctx, (void **)pp, sizeof(float) * n));
        k_narrow<<<nb(n, 256), 256, 0, ctx->stream>>>(n, ctx->d_mcc, S.f_mcc);
    }
    if (S.f_dinv_k2 != k2) {
        k_narrow<<<nb(n, 256), 256, 0, ctx->stream>>>(n, dinv, S.f_dinv);
        S.f_dinv_k2 = k2;
    }
    double *r = S.cg_r, *Ap = S.cg_Ap, *sc = S.cg_sc;
    if (warm) {
        EFE_TRY(lap_apply(ctx, phi, Ap, shift));
        k_axpy_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, 1.0, F, -1.0, Ap, r);
    } else {
        EFE_CUDA(ctx, cudaMemsetAsync(phi, 0, sizeof(double) * n, ctx->stream));
        EFE_CUDA(ctx, cudaMemcpyAsync(r, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    EFE_CUDA(ctx, cudaMemsetAsync(S.f_d, 0, sizeof(float) * n, ctx->stream));
    int total = 0;
    double hs[CG_NSC];
    double rn_prev = 0.0;
    for (int outer = 0; outer < kMaxOuter && total < max_it; ++outer) {
        double rn2;
        EFE_TRY(dot(ctx, n, r, r, rn2));
        const double rn = std::sqrt(rn2);
        if (!(rn >= thr)) break;                      // converged (or not finite: the FP64 CG reports it)
        if (outer > 0 && !(rn < 0.5 * rn_prev)) break;   // FP32 no longer gains: the FP64 CG takes over
        rn_prev = rn;
        k_narrow<<<nb(n, 256), 256, 0, ctx->stream>>>(n, r, S.f_r);
        k_set_scalar<<<1, 1, 0, ctx->stream>>>(sc, CG_THR, std::max(kInnerEta * rn, 0.5 * thr));
        k_set_scalar<<<1, 1, 0, ctx->stream>>>(sc, CG_ALPHA, 0.0);
        k_cg_update_f<<<NRED, 256, 0, ctx->stream>>>(n, sc, S.f_d, S.f_r, S.f_p, S.f_Ap, S.f_dinv, S.f_z, S.cg_part);
        k_cg_beta<<<1, 32, 0, ctx->stream>>>(S.cg_part, sc, 1);
        EFE_CUDA(ctx, cudaMemcpyAsync(S.f_p, S.f_z, sizeof(float) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        EFE_TRY(efe_check_launch(ctx, "poisson inner start"));
        EFE_CUDA(ctx, cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        bool done = hs[CG_DONE] != 0.0;
        int issued = 0;
        const int cap = max_it - total;
        while (!done && issued < cap) {
            const int blk = std::min(kCgBlock, cap - issued);
            for (int k = 0; k < blk; ++k) {
                EFE_TRY(lap_apply_f(ctx, S.f_p, S.f_Ap, (float)shift));
                k_dotp_f<<<NRED, 256, 0, ctx->stream>>>(n, S.f_p, S.f_Ap, S.cg_part);
                k_cg_alpha<<<1, 32, 0, ctx->stream>>>(S.cg_part, sc);
                k_cg_update_f<<<NRED, 256, 0, ctx->stream>>>(n, sc, S.f_d, S.f_r, S.f_p, S.f_Ap, S.f_dinv, S.f_z,
                                                             S.cg_part);
                k_cg_beta<<<1, 32, 0, ctx->stream>>>(S.cg_part, sc, 0);
                k_cg_p_f<<<nb(n, 256), 256, 0, ctx->stream>>>(n, sc, S.f_z, S.f_p);
            }
            EFE_TRY(efe_check_launch(ctx, "poisson inner iterations"));
            issued += blk;
            EFE_CUDA(ctx, cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
            EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            done = hs[CG_DONE] != 0.0;
        }
        const int inner = (int)hs[CG_IT];
        total += inner;
        // phi += d; the FP64 residual of the new phi
        k_add_correction<<<nb(n, 256), 256, 0, ctx->stream>>>(n, phi, S.f_d);
        EFE_TRY(lap_apply(ctx, phi, Ap, shift));
        k_axpy_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, 1.0, F, -1.0, Ap, r);
        EFE_TRY(efe_check_launch(ctx, "poisson refinement"));
        if (inner == 0) break;                        // no progress in FP32: the FP64 CG takes over
    }
    *iters = total;
    return EFE_OK;
}

// FE solution of -1/(4 pi) Lap phi + k2/(4 pi) phi = f (k2 = 0: Poisson), phi = 0
// on the box, with the lumped mass for the k2 term: Jacobi-preconditioned CG to
// ||r|| < tol ||F||.  warm: start from the phi passed in (else from 0).  With
// the mixed setting (efe_set_poisson_precision; by default on meshes of 2^20
// nodes or more) a refinement stage (poisson_mixed) brings the FP64 residual
// below the tolerance first; the FP64 CG then starts from its phi, checks the
// residual and iterates only if the stage stopped short.  The scalars stay on the
// device; the host reads the convergence flag once every kCgBlock iterations,
// and iterations after convergence change nothing.
static efe_status poisson(efe_ctx *ctx, const double *fq, double *phi, double *phi_q, double tol, int max_it,
                          int *iters, double *rel_res, bool warm = false, double k2 = 0.0) {
    ScfState &S = scf_state(ctx);
    const double shift = k2 / (4.0 * kPi);
    const double *dinv = S.d_dinv;
    if (shift != 0.0) {
        if (!S.d_dinv_shift) EFE_TRY(efe_alloc(ctx, (void **)&S.d_dinv_shift, sizeof(double) * ctx->n_nodes));
        if (S.shift_k2 != k2) {
            k_shift_jacobi<<<nb(ctx->n_nodes, 256), 256, 0, ctx->stream>>>(ctx->n_nodes, shift, ctx->d_mcc, S.d_dinv,
                                                                           S.d_dinv_shift);
            EFE_TRY(efe_check_launch(ctx, "k_shift_jacobi"));
            S.shift_k2 = k2;
        }
        dinv = S.d_dinv_shift;
    }
    const MeshDev &m = ctx->m;
    const long long n = ctx->n_nodes;
    Tables1D T = make_tables(ctx);
    if (!S.cg_r) {
        for (double **pp : {&S.cg_F, &S.cg_r, &S.cg_z, &S.cg_p, &S.cg_Ap})
            EFE_TRY(efe_alloc(ctx, (void **)pp, sizeof(double) * n));
        EFE_TRY(efe_alloc(ctx, (void **)&S.cg_sc, sizeof(double) * CG_NSC));
        EFE_TRY(efe_alloc(ctx, (void **)&S.cg_part, sizeof(double) * 2 * NRED));
    }
    double *F = S.cg_F, *r = S.cg_r, *z = S.cg_z, *p = S.cg_p, *Ap = S.cg_Ap, *sc = S.cg_sc;
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
    int it = 0, it_mixed = 0;
    double rr = 0.0;
    const bool mixed = ctx->poisson_mixed > 0 || (ctx->poisson_mixed < 0 && n >= (1LL << 20));
    if (mixed && bnorm > 0.0) {
        EFE_TRY(poisson_mixed(ctx, S, F, phi, warm, shift, dinv, k2, tol * bnorm, max_it, &it_mixed));
        warm = true;
    }
    if (!(bnorm > 0.0)) {
        EFE_CUDA(ctx, cudaMemsetAsync(phi, 0, sizeof(double) * n, ctx->stream));
    } else {
        // r = F - K phi0 (warm) or F (cold, phi0 = 0); z = D^-1 r; p = z
        if (warm) {
            EFE_TRY(lap_apply(ctx, phi, Ap, shift));
            k_axpy_n<<<nb(n, 256), 256, 0, ctx->stream>>>(n, 1.0, F, -1.0, Ap, r);
        } else {
            EFE_CUDA(ctx, cudaMemsetAsync(phi, 0, sizeof(double) * n, ctx->stream));
            EFE_CUDA(ctx, cudaMemcpyAsync(r, F, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        }
        k_set_scalar<<<1, 1, 0, ctx->stream>>>(sc, CG_THR, tol * bnorm);
        k_set_scalar<<<1, 1, 0, ctx->stream>>>(sc, CG_ALPHA, 0.0);
        // with alpha = 0 the update only forms z = D^-1 r and the partials of r.r, r.z
        // (p and Ap are not read)
        k_cg_update<<<NRED, 256, 0, ctx->stream>>>(n, sc, phi, r, p, Ap, dinv, z, S.cg_part);
        k_cg_beta<<<1, 32, 0, ctx->stream>>>(S.cg_part, sc, 1);
        EFE_CUDA(ctx, cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        EFE_TRY(efe_check_launch(ctx, "poisson start"));
        double hs[CG_NSC];
        EFE_CUDA(ctx, cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        rr = hs[CG_RR];
        int issued = 0;
        bool done = hs[CG_DONE] != 0.0;
        while (!done && issued < max_it) {
            const int blk = std::min(kCgBlock, max_it - issued);
            for (int k = 0; k < blk; ++k) {
                EFE_TRY(lap_apply(ctx, p, Ap, shift));
                k_dotp<<<NRED, 256, 0, ctx->stream>>>(n, p, Ap, S.cg_part);
                k_cg_alpha<<<1, 32, 0, ctx->stream>>>(S.cg_part, sc);
                k_cg_update<<<NRED, 256, 0, ctx->stream>>>(n, sc, phi, r, p, Ap, dinv, z, S.cg_part);
                k_cg_beta<<<1, 32, 0, ctx->stream>>>(S.cg_part, sc, 0);
                k_cg_p<<<nb(n, 256), 256, 0, ctx->stream>>>(n, sc, z, p);
            }
            EFE_TRY(efe_check_launch(ctx, "poisson iterations"));
            issued += blk;
            EFE_CUDA(ctx, cudaMemcpyAsync(hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
            EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            done = hs[CG_DONE] != 0.0;
        }
        it = (int)hs[CG_IT];
        rr = hs[CG_RR];
    }
    if (phi_q) EFE_TRY(cell_values(ctx, phi, nullptr, 1, nullptr, 1, phi_q));
    if (iters) *iters = it + it_mixed;
    if (rel_res) *rel_res = bnorm > 0 ? rr / bnorm : 0.0;
    return EFE_OK;
}

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

efe_status efe_set_poisson_precision(efe_ctx *ctx, efe_precision prec) {
    if (!ctx) return EFE_ERR_ARG;
    if (prec != EFE_FP64 && prec != EFE_FP32) {
        ctx->err = "efe_set_poisson_precision: EFE_FP64 or EFE_FP32";
        return EFE_ERR_ARG;
    }
    ctx->poisson_mixed = prec == EFE_FP32 ? 1 : 0;
    return EFE_OK;
}

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
    if (o->mix_history < 0 || o->mix_history > kMixMax) {
        ctx->err = "efe_scf: mix_history must be in [0, 8]";
        return EFE_ERR_ARG;
    }
    const int hist = o->mix_history;
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
           *phi2 = take(sizeof(double) * nn),
           *phi_q = take(sizeof(double) * nq), *tmp = take(sizeof(double) * nq),
           *HX = take(sizeof(double) * rows * N), *Vout = take(sizeof(double) * rows * N),
           *dlam = take(sizeof(double) * N), *hin = take(sizeof(double) * nq * HS), *hres = take(sizeof(double) * nq * HS),
           *mixpart = take(sizeof(double) * (NRED + 1) * kMixNV);
    const bool kerker = o->precond_k2 > 0.0;
    double *phik = kerker ? take(sizeof(double) * nn) : nullptr, *phik_q = kerker ? take(sizeof(double) * nq) : nullptr;
    if (!rho_in || !rho_out || !veff || !vxc || !exc || !phi || !phi2 || !phi_q || !tmp || !HX || !Vout || !dlam || !hin ||
        !hres || !mixpart || (kerker && (!phik || !phik_q))) {
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
    double maxres = 1e300;            // largest occupied residual after the last Rayleigh-Ritz
    int nh = 0;                       // history entries stored (ring of HS)
    int it = 0;
    const efe_precision prec = (efe_precision)o->precision;
    res->poisson_iters = 0;
    for (int k = 0; k < 5; ++k) res->ms_phase[k] = 0.0;
    auto tprev = std::chrono::steady_clock::now();
    auto mark = [&](int k) {
        if (!o->profile) return;
        cudaStreamSynchronize(ctx->stream);
        const auto t = std::chrono::steady_clock::now();
        res->ms_phase[k] += std::chrono::duration<double, std::milli>(t - tprev).count();
        tprev = t;
    };
    for (it = 1; it <= o->max_iter; ++it) {
        int pit = 0;
        // v_eff = v_xc[rho_in] + phi[rho_in + b]
        // each Poisson solve starts from the previous solution of the same kind
        k_add3<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_in, S.d_b, tmp);
        SCF_TRY(poisson(ctx, tmp, phi, phi_q, o->poisson_tol, 100000, &pit, nullptr, it > 1));
        res->poisson_iters += pit;
        k_lda<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_in, vxc, nullptr);
        k_add3<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, vxc, phi_q, veff);
        SCF_TRY(efe_potential_assembly(ctx, veff));
        mark(0);
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
            const int npass = std::max(1, o->passes);
            for (int ps = 0; ps < npass; ++ps) {
                if (ps > 0 && cudaMemcpyAsync(dlam, eig.data(), sizeof(double) * N, cudaMemcpyHostToDevice,
                                              ctx->stream) != cudaSuccess) {
                    cleanup();
                    return EFE_ERR_CUDA;
                }
                const double bd[3] = {eig[0], eig[N - 1], lz[2]};
                // mixed schedule: after the first iteration, bf16 passes only while the
                // occupied residuals are large (bf16_resid = 0: every pass in bf16)
                const efe_precision pp =
                    (prec == EFE_BF16 && o->bf16_resid > 0.0 && maxres <= o->bf16_resid) ? EFE_FP32 : prec;
                SCF_TRY(efe_filter(ctx, X, HX, dlam, N, o->cheb_degree, bd, pp, Vout));
                SCF_TRY(efe_rayleigh_ritz(ctx, Vout, HX, N, eig.data(), resid.data()));
                if (cudaMemcpyAsync(X, Vout, sizeof(double) * rows * N, cudaMemcpyDeviceToDevice, ctx->stream) !=
                    cudaSuccess) {
                    cleanup();
                    return EFE_ERR_CUDA;
                }
            }
        }
        mark(1);
        maxres = 0.0;
        for (int j = 0; j < std::min(nocc, N); ++j) maxres = std::max(maxres, resid[j]);
        SCF_TRY(efe_fermi(ctx, eig.data(), N, ne, kT, &mu, occ.data()));
        SCF_TRY(efe_density(ctx, X, N, occ.data(), rho_out));
        if (o->renormalize) {
            double tot;
            SCF_TRY(integrate(ctx, rho_out, nullptr, tot));
            k_scale_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, ne / tot, rho_out);
        }
        mark(2);
        // energies
        k_add3<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, rho_out, S.d_b, tmp);
        SCF_TRY(poisson(ctx, tmp, phi2, phi_q, o->poisson_tol, 100000, &pit, nullptr, it > 1));
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
        mark(3);
        if (o->log) o->log(o->log_user, it, E, F, mu, dr, dE, resid[0]);
        if (dr < o->tol_rho && dE < o->tol_e) {
            conv = true;
            break;
        }
        E_prev = E;
        have_prev = true;
        // Anderson (Walker-Ni form) on the quadrature-point densities: rings of
        // rho_in and of R = rho_out - rho_in; one pass forms the normal equations
        const int slot = nh % HS;
        cudaMemcpyAsync(hin + (size_t)slot * nq, rho_in, sizeof(double) * nq, cudaMemcpyDeviceToDevice, ctx->stream);
        k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_out, -1.0, rho_in, hres + (size_t)slot * nq);
        ++nh;
        const int have = std::min(nh, HS);           // entries, oldest first
        auto at = [&](double *base, int k) { return base + (size_t)((nh - have + k) % HS) * nq; };
        const int mm = have - 1;
        MixRing ring{};
        for (int k = 0; k < have; ++k) {
            ring.x[k] = at(hin, k);
            ring.R[k] = at(hres, k);
        }
        MixCoef gc{};
        if (mm > 0) {
            k_mix_gram<<<NRED, 256, 0, ctx->stream>>>(ctx->m, T, ring, mm, mixpart);
            k_mix_sum<<<1, 64, 0, ctx->stream>>>(NRED, mixpart, mixpart + (size_t)NRED * kMixNV);
            double hv[kMixNV];
            if (cudaMemcpyAsync(hv, mixpart + (size_t)NRED * kMixNV, sizeof(hv), cudaMemcpyDeviceToHost,
                                ctx->stream) != cudaSuccess ||
                cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
                cleanup();
                return EFE_ERR_CUDA;
            }
            std::vector<double> A(mm * mm), bvec(mm), gamma(mm, 0.0);
            for (int i = 0; i < mm; ++i) {
                for (int j = i; j < mm; ++j) A[i * mm + j] = A[j * mm + i] = hv[mix_idx(i, j)];
                bvec[i] = hv[kMixNV - kMixMax + i];
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
            for (int i = 0; i < mm; ++i) gc.g[i] = gamma[i];
        }
        k_mix_update<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, ring, mm, gc, o->mix_beta, rho_in,
                                                            kerker ? tmp : nullptr);
        if (kerker) {
            // Kerker: beta Rbar -> beta (Rbar - k2 (-Lap + k2)^-1 Rbar); phik = 4 pi (-Lap + k2)^-1 Rbar
            int kit = 0;
            SCF_TRY(poisson(ctx, tmp, phik, phik_q, o->poisson_tol, 100000, &kit, nullptr, nh > 1, o->precond_k2));
            res->poisson_iters += kit;
            k_axpy_n<<<nb(nq, 256), 256, 0, ctx->stream>>>(nq, 1.0, rho_in, -o->mix_beta * o->precond_k2 / (4.0 * kPi),
                                                           phik_q, rho_in);
        }
        mark(4);
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
