// Setup of the EFE discretisation: quadrature, cell matrices, enrichment and
// projector integrals, orthogonalization (paper Sec. II.B, Sec. III.A) and the
// per-potential assembly of the Hamiltonian blocks (Eq. KS).
#include "efe_internal.cuh"
#include "efe_funcs.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// 1D rules.  Legendre P_n and P_n' by the three-term recurrence; Gauss points
// are the roots of P_n, GLL interior points the roots of P_p' (Newton).
// ---------------------------------------------------------------------------
void legendre(int n, double x, double &P, double &dP, double &Pm1) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { P = 1.0; dP = 0.0; Pm1 = 0.0; return; }
    for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
    }
    P = p1;
    Pm1 = p0;
    dP = n * (p0 - x * p1) / (1.0 - x * x);
}

void gauss_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double P, dP, Pm1;
            legendre(n, z, P, dP, Pm1);
            double dz = P / dP;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double P, dP, Pm1;
        legendre(n, z, P, dP, Pm1);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
    }
}

void gll_rule(int p, std::vector<double> &x, std::vector<double> &w) {
    x.assign(p + 1, 0.0);
    w.assign(p + 1, 0.0);
    x[0] = -1.0;
    x[p] = 1.0;
    for (int i = 1; i < p; ++i) {
        double z = -std::cos(kPi * i / p);
        for (int it = 0; it < 100; ++it) {
            double P, dP, Pm1;
            legendre(p, z, P, dP, Pm1);
            double d2P = (2.0 * z * dP - p * (p + 1.0) * P) / (1.0 - z * z);
            double dz = dP / d2P;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
    for (int i = 0; i <= p; ++i) {
        double P, dP, Pm1;
        if (i == 0 || i == p) {
            P = (i == p) ? 1.0 : ((p % 2) ? -1.0 : 1.0);
        } else {
            legendre(p, x[i], P, dP, Pm1);
        }
        w[i] = 2.0 / (p * (p + 1.0) * P * P);
    }
}

// Lagrange polynomial a on `nodes` and its derivative at t (product forms).
double lag(const std::vector<double> &nd, int a, double t) {
    double v = 1.0;
    for (size_t b = 0; b < nd.size(); ++b)
        if ((int)b != a) v *= (t - nd[b]) / (nd[a] - nd[b]);
    return v;
}
double dlag(const std::vector<double> &nd, int a, double t) {
    double s = 0.0;
    for (size_t c = 0; c < nd.size(); ++c) {
        if ((int)c == a) continue;
        double term = 1.0 / (nd[a] - nd[c]);
        for (size_t b = 0; b < nd.size(); ++b)
            if ((int)b != a && b != c) term *= (t - nd[b]) / (nd[a] - nd[b]);
        s += term;
    }
    return s;
}

// ---------------------------------------------------------------------------
// Static projections for one (atom, cell) pair onto the cell's nodes:
//   B[l][f]   = int a_f N_l,   Kca[l][f] = 1/2 int grad a_f . grad N_l,
//   Pc[l][f]  = int beta_f N_l.
// Pairs of one colour never share a node within an atom, so += is race free.
// ---------------------------------------------------------------------------
__global__ void k_static_pairs(MeshDev m, Tables1D T, FuncParams fp, const PairInfo *pairs,
                               int p0, const int *pair_pos, const long long *sup_off,
                               const double *atoms, double *dB, double *dK, double *dP) {
    extern __shared__ double sh[];
    const int nq3 = m.nq3;
    double *F = sh;                       // nq3 x 20
    const PairInfo pr = pairs[p0 + blockIdx.x];
    const double J = 0.125 * m.h * m.h * m.h;
    const double ax = atoms[3 * pr.atom], ay = atoms[3 * pr.atom + 1], az = atoms[3 * pr.atom + 2];
    for (int q = threadIdx.x; q < nq3; q += blockDim.x) {
        double x, y, z;
        quad_point(m, T.xq, pr.cell, q, x, y, z);
        double a[4], ga[4][3], b[4];
        eval_funcs(fp, x - ax, y - ay, z - az, a, ga, b);
        int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J;
        for (int f = 0; f < 4; ++f) {
            F[q * 20 + f] = w * a[f];
            F[q * 20 + 4 + 3 * f + 0] = 0.5 * w * ga[f][0];
            F[q * 20 + 4 + 3 * f + 1] = 0.5 * w * ga[f][1];
            F[q * 20 + 4 + 3 * f + 2] = 0.5 * w * ga[f][2];
            F[q * 20 + 16 + f] = w * b[f];
        }
    }
    __syncthreads();
    const double s = 2.0 / m.h;
    const int np1 = m.np1;
    const int gbase = (int)sup_off[pr.atom];
    for (int l = threadIdx.x; l < m.ne; l += blockDim.x) {
        int pos = pair_pos[(size_t)(p0 + blockIdx.x) * m.ne + l];
        if (pos < 0) continue;
        int lx = l % np1, ly = (l / np1) % np1, lz = l / (np1 * np1);
        double accB[4] = {0, 0, 0, 0}, accK[4] = {0, 0, 0, 0}, accP[4] = {0, 0, 0, 0};
        for (int q = 0; q < nq3; ++q) {
            int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
            double bx = T.B1[qx * np1 + lx], by = T.B1[qy * np1 + ly], bz = T.B1[qz * np1 + lz];
            double N = bx * by * bz;
            double gx = s * T.D1[qx * np1 + lx] * by * bz;
            double gy = s * bx * T.D1[qy * np1 + ly] * bz;
            double gz = s * bx * by * T.D1[qz * np1 + lz];
            const double *Fq = F + q * 20;
            for (int f = 0; f < 4; ++f) {
                accB[f] += Fq[f] * N;
                accK[f] += Fq[4 + 3 * f] * gx + Fq[5 + 3 * f] * gy + Fq[6 + 3 * f] * gz;
                accP[f] += Fq[16 + f] * N;
            }
        }
        size_t g = (size_t)(gbase + pos) * 4;
        for (int f = 0; f < 4; ++f) {
            dB[g + f] += accB[f];
            dK[g + f] += accK[f];
            dP[g + f] += accP[f];
        }
    }
}

// Potential coupling for one pair: Hca[l][f] += int v a_f N_l.
// node-major copies of the coupling tables (statics on the first call, H^ca always)
// Node-major copies of the coupling entries.  nm_atom carries the atom in its
// low 29 bits and two flags: bit 30 when the entry's E is nonzero, bit 29 when
// its P_c is (E vanishes exactly outside the enrichment's one-cell dilation,
// P_c outside the projector ball), so the node kernels skip the zero halves.
__global__ void k_node_major(long long n, const int *node_ent, const int *ent_atom, const float *E32,
                             const float *P32, int statics, int *nm_atom, float *nm_E, float *nm_P) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int g = node_ent[e];
    float4 ev = make_float4(0.f, 0.f, 0.f, 0.f);
    if (E32) {
        ev = reinterpret_cast<const float4 *>(E32)[g];
        reinterpret_cast<float4 *>(nm_E)[e] = ev;
    }
    const float4 pv = reinterpret_cast<const float4 *>(P32)[g];
    if (statics) reinterpret_cast<float4 *>(nm_P)[e] = pv;
    const bool he = ev.x != 0.f || ev.y != 0.f || ev.z != 0.f || ev.w != 0.f;
    const bool hp = pv.x != 0.f || pv.y != 0.f || pv.z != 0.f || pv.w != 0.f;
    nm_atom[e] = ent_atom[g] | (he ? kNmHasE : 0) | (hp ? kNmHasP : 0);
}

__global__ void k_potential_pairs(MeshDev m, Tables1D T, FuncParams fp, const PairInfo *pairs,
                                  int p0, const int *pair_pos, const long long *sup_off,
                                  const double *atoms, const double *vq, double *dH) {
    extern __shared__ double sh[];
    const int nq3 = m.nq3;
    double *F = sh;   // nq3 x 4
    const PairInfo pr = pairs[p0 + blockIdx.x];
    const double J = 0.125 * m.h * m.h * m.h;
    const double ax = atoms[3 * pr.atom], ay = atoms[3 * pr.atom + 1], az = atoms[3 * pr.atom + 2];
    for (int q = threadIdx.x; q < nq3; q += blockDim.x) {
        double x, y, z;
        quad_point(m, T.xq, pr.cell, q, x, y, z);
        double a[4], ga[4][3], b[4];
        eval_funcs(fp, x - ax, y - ay, z - az, a, ga, b);
        int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J * vq[(size_t)pr.cell * nq3 + q];
        for (int f = 0; f < 4; ++f) F[q * 4 + f] = w * a[f];
    }
    __syncthreads();
    const int np1 = m.np1;
    const int gbase = (int)sup_off[pr.atom];
    for (int l = threadIdx.x; l < m.ne; l += blockDim.x) {
        int pos = pair_pos[(size_t)(p0 + blockIdx.x) * m.ne + l];
        if (pos < 0) continue;
        int lx = l % np1, ly = (l / np1) % np1, lz = l / (np1 * np1);
        double acc[4] = {0, 0, 0, 0};
        for (int q = 0; q < nq3; ++q) {
            int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
            double N = T.B1[qx * np1 + lx] * T.B1[qy * np1 + ly] * T.B1[qz * np1 + lz];
            for (int f = 0; f < 4; ++f) acc[f] += F[q * 4 + f] * N;
        }
        size_t g = (size_t)(gbase + pos) * 4;
        for (int f = 0; f < 4; ++f) dH[g + f] += acc[f];
    }
}

// Enriched-enriched sums over one cell for every ordered atom pair touching it:
//   A[If][Jg] = int a_If a_Jg, K = 1/2 int grad.grad, Pa[If][Jg] = int beta_If a_Jg,
//   V[If][Jg] = int v a_If a_Jg (when vq != nullptr: only V is accumulated).
__global__ void k_enriched_pairs(MeshDev m, Tables1D T, FuncParams fp, const int *cell_ptr,
                                 const int *cell_atoms, const double *atoms, const double *vq,
                                 int n_enr, double *A, double *K, double *Pa, double *V) {
    const int c = blockIdx.x;
    const int a0 = cell_ptr[c], a1 = cell_ptr[c + 1];
    if (a1 == a0) return;
    const double J = 0.125 * m.h * m.h * m.h;
    __shared__ double red[64][33];
    for (int ia = a0; ia < a1; ++ia) {
        for (int ja = a0; ja < a1; ++ja) {
            const int I = cell_atoms[ia], Jt = cell_atoms[ja];
            double acc[48];
            for (int i = 0; i < 48; ++i) acc[i] = 0.0;
            for (int q = threadIdx.x; q < m.nq3; q += blockDim.x) {
                double x, y, z;
                quad_point(m, T.xq, c, q, x, y, z);
                double aI[4], gI[4][3], bI[4], aJ[4], gJ[4][3], bJ[4];
                eval_funcs(fp, x - atoms[3 * I], y - atoms[3 * I + 1], z - atoms[3 * I + 2], aI, gI, bI);
                eval_funcs(fp, x - atoms[3 * Jt], y - atoms[3 * Jt + 1], z - atoms[3 * Jt + 2], aJ, gJ, bJ);
                int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
                double w = T.wq[qx] * T.wq[qy] * T.wq[qz] * J;
                if (vq) {
                    double wv = w * vq[(size_t)c * m.nq3 + q];
                    for (int f = 0; f < 4; ++f)
                        for (int g = 0; g < 4; ++g) acc[f * 4 + g] += wv * aI[f] * aJ[g];
                } else {
                    for (int f = 0; f < 4; ++f)
                        for (int g = 0; g < 4; ++g) {
                            acc[f * 4 + g] += w * aI[f] * aJ[g];
                            acc[16 + f * 4 + g] += 0.5 * w * (gI[f][0] * gJ[g][0] + gI[f][1] * gJ[g][1] +
                                                              gI[f][2] * gJ[g][2]);
                            acc[32 + f * 4 + g] += w * bI[f] * aJ[g];
                        }
                }
            }
            // block reduction of the 48 sums (warp shuffles, then across warps)
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            const int nv = vq ? 16 : 48;
            for (int i = 0; i < nv; ++i) {
                double v = acc[i];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) red[i][wid] = v;
            }
            __syncthreads();
            if (threadIdx.x < nv) {
                double s = 0.0;
                for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[threadIdx.x][wv];
                int i = threadIdx.x % 16, f = i / 4, g = i % 4;
                size_t idx = (size_t)(4 * I + f) * n_enr + 4 * Jt + g;
                int which = threadIdx.x / 16;
                if (vq) atomicAdd(&V[idx], s);
                else if (which == 0) atomicAdd(&A[idx], s);
                else if (which == 1) atomicAdd(&K[idx], s);
                else if (Pa) atomicAdd(&Pa[idx], s);
            }
            __syncthreads();
        }
    }
}

// C = B^T (M^cc)^-1 per support entry: C[g][f] = B[g][f] * minv[node].
__global__ void k_make_C(long long n, const int *sup_node, const double *minv, const double *B,
                         double *C) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n * 4) return;
    C[i] = B[i] * minv[sup_node[i / 4]];
}

// (B^T (M^cc)^-1 B) for the enriched block: for atom I (blockIdx.y) and a
// chunk of its support, accumulate into shared rows, then add to global.
__global__ void k_btmb(long long chunk, const long long *sup_off, const int *sup_node,
                       const double *minv, const double *B, const long long *node_ptr,
                       const int *node_ent, const int *ent_atom, int n_enr, double *out) {
    extern __shared__ double acc[];      // 4 x n_enr
    const int I = blockIdx.y;
    for (int i = threadIdx.x; i < 4 * n_enr; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    long long beg = sup_off[I] + blockIdx.x * chunk;
    long long end = min(sup_off[I + 1], beg + chunk);
    for (long long g = beg + threadIdx.x; g < end; g += blockDim.x) {
        int node = sup_node[g];
        double mi = minv[node];
        for (long long e = node_ptr[node]; e < node_ptr[node + 1]; ++e) {
            int gj = node_ent[e];
            int Jt = ent_atom[gj];
            for (int f = 0; f < 4; ++f)
                for (int h = 0; h < 4; ++h)
                    atomicAdd(&acc[f * n_enr + 4 * Jt + h], B[4 * g + f] * mi * B[4 * (size_t)gj + h]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * n_enr; i += blockDim.x) {
        double v = acc[i];
        if (v != 0.0) atomicAdd(&out[(size_t)(4 * I + i / n_enr) * n_enr + (i % n_enr)], v);
    }
}

// Products of two support tables summed over shared nodes: for atom I
// (blockIdx.y) and a chunk of its support,
//   out[4I+f][4J+h] += sum_j A1[g][f] B1[g'][h] + A2[g][f] B2[g'][h]
// with g the entry of atom I at node j and g' every entry (atom J) at j.
// Used for C H^ca + E C^T (the enriched block of H^E) and P_c C^T.
__global__ void k_support_pair_products(long long chunk, const long long *sup_off, const int *sup_node,
                                        const long long *node_ptr, const int *node_ent, const int *ent_atom,
                                        int n_enr, const double *A1, const double *B1, const double *A2,
                                        const double *B2, double *out) {
    extern __shared__ double acc[];      // 4 x n_enr
    const int I = blockIdx.y;
    for (int i = threadIdx.x; i < 4 * n_enr; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const long long beg = sup_off[I] + blockIdx.x * chunk;
    const long long end = min(sup_off[I + 1], beg + chunk);
    for (long long g = beg + threadIdx.x; g < end; g += blockDim.x) {
        const int node = sup_node[g];
        for (long long e = node_ptr[node]; e < node_ptr[node + 1]; ++e) {
            const int gj = node_ent[e];
            const int J = ent_atom[gj];
            for (int f = 0; f < 4; ++f)
                for (int h = 0; h < 4; ++h) {
                    double v = A1[4 * g + f] * B1[4 * (size_t)gj + h];
                    if (A2) v += A2[4 * g + f] * B2[4 * (size_t)gj + h];
                    atomicAdd(&acc[f * n_enr + 4 * J + h], v);
                }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * n_enr; i += blockDim.x) {
        const double v = acc[i];
        if (v != 0.0) atomicAdd(&out[(size_t)(4 * I + i / n_enr) * n_enr + (i % n_enr)], v);
    }
}

// out = A - 0.5 (X + X^T) for n x n (A symmetric): H^E_ee = H^aa - sym(C H^ca + E C^T)
__global__ void k_sub_sym(int n, const double *A, const double *X, double *out) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    out[idx] = A[idx] - 0.5 * (X[idx] + X[(size_t)j * n + i]);
}
// out = A - X (n_proj x n_enr)
__global__ void k_sub(long long n, const double *A, const double *X, double *out) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx < n) out[idx] = A[idx] - X[idx];
}

// The FE-enrichment block of H^E (Eq. Discrete_Eig_Gen_H with T):
// E = H^ac - C H^cc on the support entries.  For one (atom, cell) pair,
// subtract H_e C_cell^T from the entries of the cell's nodes; E starts as a
// copy of H^ac, and the pairs of one colour share no node.
__global__ void k_orth_coupling(MeshDev m, const PairInfo *pairs, int p0, const int *pair_pos,
                                const long long *sup_off, const double *He, const double *C, double *E) {
    extern __shared__ double Cc[];       // ne x 4
    const PairInfo pr = pairs[p0 + blockIdx.x];
    const int *pp = pair_pos + (size_t)(p0 + blockIdx.x) * m.ne;
    const long long gbase = sup_off[pr.atom];
    for (int l = threadIdx.x; l < m.ne; l += blockDim.x) {
        const int pos = pp[l];
        for (int f = 0; f < 4; ++f) Cc[4 * l + f] = pos >= 0 ? C[4 * (gbase + pos) + f] : 0.0;
    }
    __syncthreads();
    const double *H = He + (size_t)pr.cell * m.ne * m.ne;
    for (int l = threadIdx.x; l < m.ne; l += blockDim.x) {
        const int pos = pp[l];
        if (pos < 0) continue;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        for (int l2 = 0; l2 < m.ne; ++l2) {
            const double h = H[(size_t)l2 * m.ne + l];   // H_e is symmetric: coalesced over l
            a0 += h * Cc[4 * l2];
            a1 += h * Cc[4 * l2 + 1];
            a2 += h * Cc[4 * l2 + 2];
            a3 += h * Cc[4 * l2 + 3];
        }
        double *e = E + 4 * (gbase + pos);
        e[0] -= a0;
        e[1] -= a1;
        e[2] -= a2;
        e[3] -= a3;
    }
}

// Cell Hamiltonians H_e = 1/2 K_e + V_e with V_e by sum factorisation of
//   V[(az,ay,ax),(bz,by,bx)] = J sum_q v(q) prod_axes w B1 B1.
// One block per cell; a thread owns (az,bz,ay,by) tuples.
__global__ void k_cell_hamiltonian(MeshDev m, Tables1D T, const double *vq, const double *Khalf,
                                   double *He, float *He32) {
    extern __shared__ double sh[];
    const int nq = m.nq, np1 = m.np1, ne = m.ne, nq3 = m.nq3;
    double *wv = sh;                          // nq3
    double *BB = wv + nq3;                    // nq x np1 x np1 : w_q B1[q,a] B1[q,b]
    double *U = BB + nq * np1 * np1;          // (np1*np1) x (nq*nq)
    const int c = blockIdx.x;
    for (int q = threadIdx.x; q < nq3; q += blockDim.x) wv[q] = vq[(size_t)c * nq3 + q];
    for (int i = threadIdx.x; i < nq * np1 * np1; i += blockDim.x) {
        int q = i / (np1 * np1), a = (i / np1) % np1, b = i % np1;
        BB[i] = T.wq[q] * T.B1[q * np1 + a] * T.B1[q * np1 + b];
    }
    __syncthreads();
    const int nab = np1 * np1, nqq = nq * nq;
    for (int i = threadIdx.x; i < nab * nqq; i += blockDim.x) {
        int ab = i / nqq, yx = i % nqq;
        double s = 0.0;
        for (int qz = 0; qz < nq; ++qz) s += wv[qz * nqq + yx] * BB[qz * nab + ab];
        U[i] = s;
    }
    __syncthreads();
    const double J = 0.125 * m.h * m.h * m.h;
    for (int t = threadIdx.x; t < nab * nab; t += blockDim.x) {
        int zab = t / nab, yab = t % nab;   // (az,bz), (ay,by)
        int az = zab / np1, bz = zab % np1, ay = yab / np1, by = yab % np1;
        double W[EFE_MAXNQ];
        for (int qx = 0; qx < nq; ++qx) {
            double s = 0.0;
            for (int qy = 0; qy < nq; ++qy) s += U[zab * nqq + qy * nq + qx] * BB[qy * nab + yab];
            W[qx] = s;
        }
        for (int ax = 0; ax < np1; ++ax) {
            int row = (az * np1 + ay) * np1 + ax;
            for (int bx = 0; bx < np1; ++bx) {
                double s = 0.0;
                for (int qx = 0; qx < nq; ++qx) s += W[qx] * BB[qx * nab + ax * np1 + bx];
                int col = (bz * np1 + by) * np1 + bx;
                double v = J * s + Khalf[(size_t)row * ne + col];
                size_t o = (size_t)c * ne * ne + (size_t)row * ne + col;
                He[o] = v;
                if (He32) He32[o] = (float)v;
            }
        }
    }
}

__global__ void k_to_float(long long n, const double *a, float *b) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}
__global__ void k_copy(long long n, const double *a, double *b) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------------------
efe_status efe_build_tables(efe_ctx *ctx) {
    MeshDev &m = ctx->m;
    gll_rule(m.p, ctx->xg, ctx->wg);
    gauss_rule(m.nq, ctx->xq, ctx->wq);
    ctx->B1.assign((size_t)m.nq * m.np1, 0.0);
    ctx->D1.assign((size_t)m.nq * m.np1, 0.0);
    for (int q = 0; q < m.nq; ++q)
        for (int a = 0; a < m.np1; ++a) {
            ctx->B1[q * m.np1 + a] = lag(ctx->xg, a, ctx->xq[q]);
            ctx->D1[q * m.np1 + a] = dlag(ctx->xg, a, ctx->xq[q]);
        }
    // exact 1D mass and stiffness on [-1, 1] (Gauss, nq >= p + 1)
    const int np1 = m.np1;
    std::vector<double> M1(np1 * np1, 0.0), K1(np1 * np1, 0.0);
    for (int a = 0; a < np1; ++a)
        for (int b = 0; b < np1; ++b)
            for (int q = 0; q < m.nq; ++q) {
                M1[a * np1 + b] += ctx->wq[q] * ctx->B1[q * np1 + a] * ctx->B1[q * np1 + b];
                K1[a * np1 + b] += ctx->wq[q] * ctx->D1[q * np1 + a] * ctx->D1[q * np1 + b];
            }
    // 1/2 K_e = 1/2 (h/2) (K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1)
    const int ne = m.ne;
    std::vector<double> Kh((size_t)ne * ne);
    for (int r = 0; r < ne; ++r) {
        int ax = r % np1, ay = (r / np1) % np1, az = r / (np1 * np1);
        for (int c = 0; c < ne; ++c) {
            int bx = c % np1, by = (c / np1) % np1, bz = c / (np1 * np1);
            double v = K1[ax * np1 + bx] * M1[ay * np1 + by] * M1[az * np1 + bz] +
                       M1[ax * np1 + bx] * K1[ay * np1 + by] * M1[az * np1 + bz] +
                       M1[ax * np1 + bx] * M1[ay * np1 + by] * K1[az * np1 + bz];
            Kh[(size_t)r * ne + c] = 0.5 * (0.5 * m.h) * v;
        }
    }
    // GLL-lumped M^cc: per axis the summed 1D weights, product over axes
    auto axis_mass = [&](int ncell) {
        std::vector<double> w1(ncell * m.p + 1, 0.0);
        for (int k = 0; k < ncell; ++k)
            for (int a = 0; a <= m.p; ++a) w1[k * m.p + a] += 0.5 * m.h * ctx->wg[a];
        return w1;
    };
    auto mx = axis_mass(m.nx), my = axis_mass(m.ny), mz = axis_mass(m.nz);
    std::vector<double> mcc(ctx->n_nodes), minv(ctx->n_nodes);
    for (int iz = 0; iz < m.Gz; ++iz)
        for (int iy = 0; iy < m.Gy; ++iy)
            for (int ix = 0; ix < m.Gx; ++ix) {
                size_t n = ((size_t)iz * m.Gy + iy) * m.Gx + ix;
                double v = mx[ix] * my[iy] * mz[iz];
                bool interior = ix > 0 && iy > 0 && iz > 0 && ix < m.Gx - 1 && iy < m.Gy - 1 && iz < m.Gz - 1;
                mcc[n] = interior ? v : 0.0;
                minv[n] = interior ? 1.0 / v : 0.0;
            }
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_Khat, sizeof(double) * ne * ne));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_mcc, sizeof(double) * ctx->n_nodes));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_minv, sizeof(double) * ctx->n_nodes));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_Khat, Kh.data(), sizeof(double) * ne * ne, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_mcc, mcc.data(), sizeof(double) * ctx->n_nodes, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_minv, minv.data(), sizeof(double) * ctx->n_nodes, cudaMemcpyHostToDevice));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_B1, sizeof(double) * m.nq * np1));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_D1, sizeof(double) * m.nq * np1));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_wq, sizeof(double) * m.nq));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_B1, ctx->B1.data(), sizeof(double) * m.nq * np1, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_D1, ctx->D1.data(), sizeof(double) * m.nq * np1, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_wq, ctx->wq.data(), sizeof(double) * m.nq, cudaMemcpyHostToDevice));
    return EFE_OK;
}

// Supports, pairs, node CSR and the static integrals.
efe_status efe_static_integrals(efe_ctx *ctx) {
    const MeshDev &m = ctx->m;
    const int na = ctx->natoms;
    const bool any = ctx->enrich || ctx->nonlocal;
    ctx->sup_off.assign(na + 1, 0);
    ctx->pair_colour_off.assign(9, 0);
    if (!any || na == 0) return EFE_OK;
    // Support cells of an atom: the cells that meet the projector ball
    // (r <= rtrunc) and, with enrichment, the cells that meet the enrichment
    // ball (r <= r_end) together with every cell sharing a node with one of
    // them.  C is nonzero only at nodes of the first kind of cell, so the
    // FE-enrichment block of H^E, E = H^ac - C H^cc, is nonzero only at nodes of
    // the cells around them: the support lists carry every nonzero of E.
    const double Re = ctx->enrich ? ctx->r0 * (1.0 + 1.0 / ctx->t) : -1.0;
    const double Rp = ctx->nonlocal ? ctx->rtrunc : -1.0;
    const double Rmax = std::max(Re, Rp);
    std::vector<std::vector<int>> atom_cells(na);
    std::vector<int> mark(ctx->n_nodes, -1);
    std::vector<int> sup_node;
    std::vector<std::vector<int>> cell_atoms(m.nx * m.ny * m.nz);
    for (int I = 0; I < na; ++I) {
        const double *X = &ctx->xyz[3 * I];
        int lo[3], hi[3], nc[3] = {m.nx, m.ny, m.nz};
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::max(0, (int)std::floor((X[d] - Rmax) / m.h) - 2);
            hi[d] = std::min(nc[d] - 1, (int)std::floor((X[d] + Rmax) / m.h) + 2);
        }
        auto meets = [&](int cx, int cy, int cz, double R) {
            if (R < 0.0) return false;
            double d2 = 0.0;
            const int cc[3] = {cx, cy, cz};
            for (int d = 0; d < 3; ++d) {
                double a = cc[d] * m.h, b = a + m.h;
                double qd = std::min(std::max(X[d], a), b) - X[d];
                d2 += qd * qd;
            }
            return d2 <= R * R;
        };
        for (int cz = lo[2]; cz <= hi[2]; ++cz)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
                for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                    bool in = meets(cx, cy, cz, Rp);
                    for (int dz = -1; dz <= 1 && !in; ++dz)
                        for (int dy = -1; dy <= 1 && !in; ++dy)
                            for (int dx = -1; dx <= 1 && !in; ++dx) {
                                const int ax = cx + dx, ay = cy + dy, az = cz + dz;
                                if (ax < 0 || ay < 0 || az < 0 || ax >= m.nx || ay >= m.ny || az >= m.nz) continue;
                                in = meets(ax, ay, az, Re);
                            }
                    if (in) {
                        int c = (cz * m.ny + cy) * m.nx + cx;
                        atom_cells[I].push_back(c);
                        cell_atoms[c].push_back(I);
                    }
                }
        // support nodes: interior nodes of those cells, sorted
        std::vector<int> nodes;
        for (int c : atom_cells[I]) {
            int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
            for (int l = 0; l < m.ne; ++l) {
                int lx = l % m.np1, ly = (l / m.np1) % m.np1, lz = l / (m.np1 * m.np1);
                int ix = cx * m.p + lx, iy = cy * m.p + ly, iz = cz * m.p + lz;
                if (ix == 0 || iy == 0 || iz == 0 || ix == m.Gx - 1 || iy == m.Gy - 1 || iz == m.Gz - 1) continue;
                int n = (iz * m.Gy + iy) * m.Gx + ix;
                if (mark[n] == -2) continue;
                mark[n] = -2;
                nodes.push_back(n);
            }
        }
        std::sort(nodes.begin(), nodes.end());
        for (int n : nodes) mark[n] = -1;
        ctx->sup_off[I + 1] = ctx->sup_off[I] + (long long)nodes.size();
        sup_node.insert(sup_node.end(), nodes.begin(), nodes.end());
    }
    ctx->sup_total = ctx->sup_off[na];
    std::vector<int> ent_atom(ctx->sup_total);
    for (int I = 0; I < na; ++I)
        for (long long g = ctx->sup_off[I]; g < ctx->sup_off[I + 1]; ++g) ent_atom[g] = I;
    // node CSR
    std::vector<long long> node_ptr(ctx->n_nodes + 1, 0);
    for (long long g = 0; g < ctx->sup_total; ++g) node_ptr[sup_node[g] + 1]++;
    ctx->n_support_nodes = 0;
    for (long long n = 0; n < ctx->n_nodes; ++n) {
        if (node_ptr[n + 1] > 0) ++ctx->n_support_nodes;
        node_ptr[n + 1] += node_ptr[n];
    }
    std::vector<int> node_ent(ctx->sup_total);
    {
        std::vector<long long> fill(node_ptr.begin(), node_ptr.end() - 1);
        for (long long g = 0; g < ctx->sup_total; ++g) node_ent[fill[sup_node[g]]++] = (int)g;
    }
    // pairs, grouped by cell colour; local node -> support position
    std::vector<std::vector<PairInfo>> bycol(8);
    for (int I = 0; I < na; ++I)
        for (int c : atom_cells[I]) {
            int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
            bycol[(cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2)].push_back({I, c});
        }
    ctx->pairs.clear();
    for (int k = 0; k < 8; ++k) {
        ctx->pair_colour_off[k] = (int)ctx->pairs.size();
        ctx->pairs.insert(ctx->pairs.end(), bycol[k].begin(), bycol[k].end());
    }
    ctx->pair_colour_off[8] = (int)ctx->pairs.size();
    const size_t np = ctx->pairs.size();
    std::vector<int> pair_pos(np * m.ne, -1);
    for (size_t k = 0; k < np; ++k) {
        const PairInfo pr = ctx->pairs[k];
        const int *sn = sup_node.data() + ctx->sup_off[pr.atom];
        const long long cnt = ctx->sup_off[pr.atom + 1] - ctx->sup_off[pr.atom];
        int cx = pr.cell % m.nx, cy = (pr.cell / m.nx) % m.ny, cz = pr.cell / (m.nx * m.ny);
        for (int l = 0; l < m.ne; ++l) {
            int lx = l % m.np1, ly = (l / m.np1) % m.np1, lz = l / (m.np1 * m.np1);
            int n = ((cz * m.p + lz) * m.Gy + (cy * m.p + ly)) * m.Gx + (cx * m.p + lx);
            const int *it = std::lower_bound(sn, sn + cnt, n);
            if (it != sn + cnt && *it == n) pair_pos[k * m.ne + l] = (int)(it - sn);
        }
    }
    // cell -> atoms CSR
    std::vector<int> cptr(cell_atoms.size() + 1, 0), cat;
    for (size_t c = 0; c < cell_atoms.size(); ++c) {
        cptr[c + 1] = cptr[c] + (int)cell_atoms[c].size();
        cat.insert(cat.end(), cell_atoms[c].begin(), cell_atoms[c].end());
    }
    // upload
    const size_t S = (size_t)ctx->sup_total;
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_sup_node, sizeof(int) * std::max<size_t>(S, 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_ent_atom, sizeof(int) * std::max<size_t>(S, 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_node_ent, sizeof(int) * std::max<size_t>(S, 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_node_ptr, sizeof(long long) * (ctx->n_nodes + 1)));
    for (double **p : {&ctx->d_C, &ctx->d_B, &ctx->d_Kca, &ctx->d_Hca, &ctx->d_Pc}) {
        EFE_TRY(efe_alloc(ctx, (void **)p, sizeof(double) * 4 * std::max<size_t>(S, 1)));
        EFE_CUDA(ctx, cudaMemset(*p, 0, sizeof(double) * 4 * std::max<size_t>(S, 1)));
    }
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_pairs, sizeof(PairInfo) * std::max<size_t>(np, 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_pair_pos, sizeof(int) * std::max<size_t>(np * m.ne, 1)));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_cell_atom_ptr, sizeof(int) * cptr.size()));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_cell_atoms, sizeof(int) * std::max<size_t>(cat.size(), 1)));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_sup_node, sup_node.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_ent_atom, ent_atom.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_node_ent, node_ent.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_node_ptr, node_ptr.data(), sizeof(long long) * (ctx->n_nodes + 1),
                             cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_pairs, ctx->pairs.data(), sizeof(PairInfo) * np, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_pair_pos, pair_pos.data(), sizeof(int) * np * m.ne, cudaMemcpyHostToDevice));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_cell_atom_ptr, cptr.data(), sizeof(int) * cptr.size(), cudaMemcpyHostToDevice));
    if (!cat.empty())
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_cell_atoms, cat.data(), sizeof(int) * cat.size(), cudaMemcpyHostToDevice));
    EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_sup_off, sizeof(long long) * (na + 1)));
    EFE_CUDA(ctx, cudaMemcpy(ctx->d_sup_off, ctx->sup_off.data(), sizeof(long long) * (na + 1), cudaMemcpyHostToDevice));
    long long *d_supoff = ctx->d_sup_off;

    // static pair projections, colour by colour
    Tables1D T = make_tables(ctx);
    FuncParams fp = make_fp(ctx);
    size_t shm = sizeof(double) * m.nq3 * 20;
    EFE_CUDA(ctx, cudaFuncSetAttribute(k_static_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    for (int k = 0; k < 8; ++k) {
        int n = ctx->pair_colour_off[k + 1] - ctx->pair_colour_off[k];
        if (!n) continue;
        k_static_pairs<<<n, 256, shm, ctx->stream>>>(m, T, fp, ctx->d_pairs, ctx->pair_colour_off[k],
                                                     ctx->d_pair_pos, d_supoff, ctx->d_atoms, ctx->d_B,
                                                     ctx->d_Kca, ctx->d_Pc);
        EFE_TRY(efe_check_launch(ctx, "k_static_pairs"));
    }
    const int ne_ = ctx->n_enr;
    if (ctx->enrich) {
        const size_t E2 = (size_t)ne_ * ne_;
        for (double **p : {&ctx->d_Aee, &ctx->d_Kaa, &ctx->d_Haa, &ctx->d_Mee}) {
            EFE_TRY(efe_alloc(ctx, (void **)p, sizeof(double) * E2));
            EFE_CUDA(ctx, cudaMemset(*p, 0, sizeof(double) * E2));
        }
        if (ctx->nonlocal) {
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_Pa, sizeof(double) * ctx->n_proj * ne_));
            EFE_CUDA(ctx, cudaMemset(ctx->d_Pa, 0, sizeof(double) * ctx->n_proj * ne_));
        }
        k_enriched_pairs<<<m.nx * m.ny * m.nz, 128, 0, ctx->stream>>>(
            m, T, fp, ctx->d_cell_atom_ptr, ctx->d_cell_atoms, ctx->d_atoms, nullptr, ne_, ctx->d_Aee,
            ctx->d_Kaa, ctx->nonlocal ? ctx->d_Pa : nullptr, nullptr);
        EFE_TRY(efe_check_launch(ctx, "k_enriched_pairs"));
        k_make_C<<<nblk(S * 4, 256), 256, 0, ctx->stream>>>((long long)S, ctx->d_sup_node, ctx->d_minv,
                                                            ctx->d_B, ctx->d_C);
        EFE_TRY(efe_check_launch(ctx, "k_make_C"));
        // M^ee = A_ee - B^T (M^cc)^-1 B
        double *d_btmb = nullptr;
        EFE_TRY(efe_alloc(ctx, (void **)&d_btmb, sizeof(double) * E2));
        EFE_CUDA(ctx, cudaMemset(d_btmb, 0, sizeof(double) * E2));
        long long maxsup = 0;
        for (int I = 0; I < na; ++I) maxsup = std::max(maxsup, ctx->sup_off[I + 1] - ctx->sup_off[I]);
        const long long chunk = 4096;
        size_t shb = sizeof(double) * 4 * ne_;
        EFE_CUDA(ctx, cudaFuncSetAttribute(k_btmb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb));
        dim3 g((unsigned)((maxsup + chunk - 1) / chunk), na);
        k_btmb<<<g, 256, shb, ctx->stream>>>(chunk, d_supoff, ctx->d_sup_node, ctx->d_minv, ctx->d_B,
                                             ctx->d_node_ptr, ctx->d_node_ent, ctx->d_ent_atom, ne_, d_btmb);
        EFE_TRY(efe_check_launch(ctx, "k_btmb"));
        std::vector<double> A(E2), BtB(E2);
        EFE_CUDA(ctx, cudaMemcpyAsync(A.data(), ctx->d_Aee, sizeof(double) * E2, cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaMemcpyAsync(BtB.data(), d_btmb, sizeof(double) * E2, cudaMemcpyDeviceToHost, ctx->stream));
        EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cudaFree(d_btmb);
        std::vector<double> Mee(E2);
        for (int i = 0; i < ne_; ++i)
            for (int j = 0; j < ne_; ++j) {
                double a = A[(size_t)i * ne_ + j] - BtB[(size_t)i * ne_ + j];
                double b = A[(size_t)j * ne_ + i] - BtB[(size_t)j * ne_ + i];
                Mee[(size_t)i * ne_ + j] = 0.5 * (a + b);
            }
        // atom blocks: Cholesky (SPD check) and inverse by Gauss-Jordan
        std::vector<double> blk(16 * na), binv(16 * na);
        for (int I = 0; I < na; ++I) {
            double Mb[16], L[16] = {0};
            for (int f = 0; f < 4; ++f)
                for (int g2 = 0; g2 < 4; ++g2) Mb[f * 4 + g2] = Mee[(size_t)(4 * I + f) * ne_ + 4 * I + g2];
            for (int j = 0; j < 4; ++j) {
                double s = Mb[j * 4 + j];
                for (int k = 0; k < j; ++k) s -= L[j * 4 + k] * L[j * 4 + k];
                if (!(s > 0.0)) {
                    char buf[160];
                    snprintf(buf, sizeof buf, "M^ee block of atom %d is not positive definite", I);
                    ctx->err = buf;
                    return EFE_ERR_NOT_SPD;
                }
                L[j * 4 + j] = std::sqrt(s);
                for (int i = j + 1; i < 4; ++i) {
                    double t = Mb[i * 4 + j];
                    for (int k = 0; k < j; ++k) t -= L[i * 4 + k] * L[j * 4 + k];
                    L[i * 4 + j] = t / L[j * 4 + j];
                }
            }
            double aug[4][8];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 8; ++j) aug[i][j] = j < 4 ? Mb[i * 4 + j] : (j - 4 == i ? 1.0 : 0.0);
            for (int col = 0; col < 4; ++col) {
                int piv = col;
                for (int r = col + 1; r < 4; ++r)
                    if (std::fabs(aug[r][col]) > std::fabs(aug[piv][col])) piv = r;
                for (int j = 0; j < 8; ++j) std::swap(aug[col][j], aug[piv][j]);
                double d = aug[col][col];
                for (int j = 0; j < 8; ++j) aug[col][j] /= d;
                for (int r = 0; r < 4; ++r)
                    if (r != col) {
                        double f = aug[r][col];
                        for (int j = 0; j < 8; ++j) aug[r][j] -= f * aug[col][j];
                    }
            }
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    blk[16 * I + i * 4 + j] = Mb[i * 4 + j];
                    binv[16 * I + i * 4 + j] = aug[i][4 + j];
                }
        }
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_Mee, Mee.data(), sizeof(double) * E2, cudaMemcpyHostToDevice));
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_Mblk, sizeof(double) * 16 * na));
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_Mblk_inv, sizeof(double) * 16 * na));
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_Mblk, blk.data(), sizeof(double) * 16 * na, cudaMemcpyHostToDevice));
        EFE_CUDA(ctx, cudaMemcpy(ctx->d_Mblk_inv, binv.data(), sizeof(double) * 16 * na, cudaMemcpyHostToDevice));
        if (ctx->nonlocal) {
            // projector overlaps of the orthogonalized functions: P^E = P_a - P_c C^T
            const size_t PE = (size_t)ctx->n_proj * ne_;
            double *d_pct = nullptr;
            EFE_TRY(efe_alloc(ctx, (void **)&d_pct, sizeof(double) * PE));
            EFE_CUDA(ctx, cudaMemset(d_pct, 0, sizeof(double) * PE));
            EFE_CUDA(ctx, cudaFuncSetAttribute(k_support_pair_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)shb));
            k_support_pair_products<<<g, 256, shb, ctx->stream>>>(chunk, d_supoff, ctx->d_sup_node, ctx->d_node_ptr,
                                                                  ctx->d_node_ent, ctx->d_ent_atom, ne_, ctx->d_Pc,
                                                                  ctx->d_C, nullptr, nullptr, d_pct);
            EFE_TRY(efe_check_launch(ctx, "k_support_pair_products(PcC)"));
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_PE, sizeof(double) * PE));
            k_sub<<<nblk((long long)PE, 256), 256, 0, ctx->stream>>>((long long)PE, ctx->d_Pa, d_pct, ctx->d_PE);
            EFE_TRY(efe_check_launch(ctx, "k_sub(PE)"));
            EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(d_pct);
        }
    }
    return EFE_OK;
}

// Per-potential assembly: cell Hamiltonians and the potential coupling blocks.
efe_status efe_potential_assembly(efe_ctx *ctx, const double *veff_q) {
    const MeshDev &m = ctx->m;
    const long long ncell = (long long)m.nx * m.ny * m.nz;
    const size_t he = (size_t)ncell * m.ne * m.ne;
    if (!ctx->d_He) {
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_He, sizeof(double) * he));
        EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_He32, sizeof(float) * he));
    }
    Tables1D T = make_tables(ctx);
    size_t shm = sizeof(double) * (m.nq3 + m.nq * m.np1 * m.np1 + m.np1 * m.np1 * m.nq * m.nq);
    EFE_CUDA(ctx, cudaFuncSetAttribute(k_cell_hamiltonian, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_cell_hamiltonian<<<(unsigned)ncell, 256, shm, ctx->stream>>>(m, T, veff_q, ctx->d_Khat, ctx->d_He,
                                                                  ctx->d_He32);
    EFE_TRY(efe_check_launch(ctx, "k_cell_hamiltonian"));
    ctx->he16_valid = false;
    if (ctx->enrich && ctx->natoms) {
        const long long S4 = 4 * ctx->sup_total;
        k_copy<<<nblk(S4, 256), 256, 0, ctx->stream>>>(S4, ctx->d_Kca, ctx->d_Hca);
        long long *d_supoff = ctx->d_sup_off;
        FuncParams fp = make_fp(ctx);
        size_t shp = sizeof(double) * m.nq3 * 4;
        for (int k = 0; k < 8; ++k) {
            int n = ctx->pair_colour_off[k + 1] - ctx->pair_colour_off[k];
            if (!n) continue;
            k_potential_pairs<<<n, 256, shp, ctx->stream>>>(m, T, fp, ctx->d_pairs, ctx->pair_colour_off[k],
                                                            ctx->d_pair_pos, d_supoff, ctx->d_atoms, veff_q,
                                                            ctx->d_Hca);
            EFE_TRY(efe_check_launch(ctx, "k_potential_pairs"));
        }
        const size_t E2 = (size_t)ctx->n_enr * ctx->n_enr;
        EFE_CUDA(ctx, cudaMemcpyAsync(ctx->d_Haa, ctx->d_Kaa, sizeof(double) * E2, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
        k_enriched_pairs<<<(unsigned)ncell, 128, 0, ctx->stream>>>(
            m, T, fp, ctx->d_cell_atom_ptr, ctx->d_cell_atoms, ctx->d_atoms, veff_q, ctx->n_enr, nullptr,
            nullptr, nullptr, ctx->d_Haa);
        EFE_TRY(efe_check_launch(ctx, "k_enriched_pairs(v)"));
        // the blocks of H^E that touch the enriched rows, in FP64:
        //   E = H^ac - C H^cc (support entries), H^E_ee = H^aa - C H^ca - E C^T
        if (!ctx->d_E) {
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_E, sizeof(double) * S4));
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_HEee, sizeof(double) * 2 * E2));
        }
        EFE_CUDA(ctx, cudaMemcpyAsync(ctx->d_E, ctx->d_Hca, sizeof(double) * S4, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
        const size_t sho = sizeof(double) * 4 * m.ne;
        for (int k = 0; k < 8; ++k) {
            int n = ctx->pair_colour_off[k + 1] - ctx->pair_colour_off[k];
            if (!n) continue;
            k_orth_coupling<<<n, 256, sho, ctx->stream>>>(m, ctx->d_pairs, ctx->pair_colour_off[k], ctx->d_pair_pos,
                                                          d_supoff, ctx->d_He, ctx->d_C, ctx->d_E);
            EFE_TRY(efe_check_launch(ctx, "k_orth_coupling"));
        }
        double *acc = ctx->d_HEee + E2;       // second half: the products, summed
        EFE_CUDA(ctx, cudaMemsetAsync(acc, 0, sizeof(double) * E2, ctx->stream));
        long long maxsup = 0;
        for (int I = 0; I < ctx->natoms; ++I) maxsup = std::max(maxsup, ctx->sup_off[I + 1] - ctx->sup_off[I]);
        const long long chunk = 4096;
        const size_t shb = sizeof(double) * 4 * ctx->n_enr;
        EFE_CUDA(ctx, cudaFuncSetAttribute(k_support_pair_products, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)shb));
        dim3 gp((unsigned)std::max<long long>(1, (maxsup + chunk - 1) / chunk), ctx->natoms);
        k_support_pair_products<<<gp, 256, shb, ctx->stream>>>(chunk, d_supoff, ctx->d_sup_node, ctx->d_node_ptr,
                                                               ctx->d_node_ent, ctx->d_ent_atom, ctx->n_enr, ctx->d_C,
                                                               ctx->d_Hca, ctx->d_E, ctx->d_C, acc);
        EFE_TRY(efe_check_launch(ctx, "k_support_pair_products(HEee)"));
        k_sub_sym<<<nblk((long long)E2, 256), 256, 0, ctx->stream>>>(ctx->n_enr, ctx->d_Haa, acc, ctx->d_HEee);
        EFE_TRY(efe_check_launch(ctx, "k_sub_sym"));
    }
    if ((ctx->enrich || ctx->nonlocal) && ctx->natoms) {
        const long long S4 = 4 * std::max<long long>(ctx->sup_total, 1);
        const bool first = ctx->d_Pc32 == nullptr;
        if (first) {
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_E32, sizeof(float) * S4));
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_Pc32, sizeof(float) * S4));
            k_to_float<<<nblk(S4, 256), 256, 0, ctx->stream>>>(S4, ctx->d_Pc, ctx->d_Pc32);
        }
        if (ctx->enrich) k_to_float<<<nblk(S4, 256), 256, 0, ctx->stream>>>(S4, ctx->d_E, ctx->d_E32);
        EFE_TRY(efe_check_launch(ctx, "k_to_float"));
        // node-major copies: entry e of the node CSR carries its atom and coefficients
        const long long ns = std::max<long long>(ctx->sup_total, 1);
        if (first) {
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_nm_atom, sizeof(int) * ns));
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_nm_E32, sizeof(float) * 4 * ns));
            EFE_TRY(efe_alloc(ctx, (void **)&ctx->d_nm_P32, sizeof(float) * 4 * ns));
        }
        if (ctx->sup_total > 0) {
            k_node_major<<<nblk(ctx->sup_total, 256), 256, 0, ctx->stream>>>(
                ctx->sup_total, ctx->d_node_ent, ctx->d_ent_atom, ctx->enrich ? ctx->d_E32 : nullptr, ctx->d_Pc32,
                first ? 1 : 0, ctx->d_nm_atom, ctx->d_nm_E32, ctx->d_nm_P32);
            EFE_TRY(efe_check_launch(ctx, "k_node_major"));
        }
    }
    ctx->have_potential = true;
    return EFE_OK;
}
