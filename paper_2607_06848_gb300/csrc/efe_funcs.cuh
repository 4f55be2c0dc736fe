// Device helpers shared by the setup and SCF translation units: quadrature
// tables and the enrichment / projector functions of one atom at a point
// (paper Sec. II.B; projector form as documented in include/efe.h).
#pragma once

#include "efe_internal.cuh"

namespace efe_dev {

constexpr double kPi = 3.14159265358979323846;

struct FuncParams {
    double alpha, r0, t, rc, rtrunc;
    int enrich, nonlocal;
};

__device__ inline void cutoff_dev(double r, double r0, double t, double &h, double &dh) {
    double s = (r - r0) * t / r0;
    if (s <= 0.0) { h = 1.0; dh = 0.0; return; }
    if (s >= 1.0) { h = 0.0; dh = 0.0; return; }
    double u = exp(-1.0 / (1.0 - s));
    double w = exp(-1.0 / s);
    double du = -u / ((1.0 - s) * (1.0 - s));
    double dw = w / (s * s);
    double den = u + w;
    h = u / den;
    dh = (du * w - u * dw) / (den * den) * (t / r0);
}

// a[4] values, ga[4][3] gradients, beta[4] projector values at displacement d.
__device__ inline void eval_funcs(const FuncParams &fp, double dx, double dy, double dz,
                                  double a[4], double ga[4][3], double beta[4]) {
    const double Y00 = 0.28209479177387814;   // 1/sqrt(4 pi)
    const double Y1C = 0.48860251190291992;   // sqrt(3/(4 pi))
    double r2 = dx * dx + dy * dy + dz * dz;
    double r = sqrt(r2);
    double d[3] = {dx, dy, dz};
    if (fp.enrich) {
        double g = exp(-fp.alpha * r2);
        double h, dh;
        cutoff_dev(r, fp.r0, fp.t, h, dh);
        double f = g * h;
        double fpr = g * ((r > 0.0 ? dh / r : 0.0) - 2.0 * fp.alpha * h);   // f'(r)/r
        a[0] = Y00 * f;
        for (int k = 0; k < 3; ++k) ga[0][k] = Y00 * fpr * d[k];
        for (int m = 0; m < 3; ++m) {
            a[1 + m] = Y1C * d[m] * f;
            for (int k = 0; k < 3; ++k) ga[1 + m][k] = Y1C * d[m] * fpr * d[k];
            ga[1 + m][m] += Y1C * f;
        }
    } else {
        for (int f = 0; f < 4; ++f) { a[f] = 0.0; ga[f][0] = ga[f][1] = ga[f][2] = 0.0; }
    }
    if (fp.nonlocal) {
        double g = (r2 > fp.rtrunc * fp.rtrunc) ? 0.0 : exp(-r2 / (2.0 * fp.rc * fp.rc));
        double As = pow(kPi * fp.rc * fp.rc, -0.75);
        double Ap = As * sqrt(2.0) / fp.rc;
        beta[0] = As * g;
        for (int m = 0; m < 3; ++m) beta[1 + m] = Ap * d[m] * g;
    } else {
        beta[0] = beta[1] = beta[2] = beta[3] = 0.0;
    }
}

__device__ inline void quad_point(const MeshDev &m, const double *xq, int c, int q, double &x,
                                  double &y, double &z) {
    int cx = c % m.nx, cy = (c / m.nx) % m.ny, cz = c / (m.nx * m.ny);
    int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
    x = cx * m.h + 0.5 * m.h * (xq[qx] + 1.0);
    y = cy * m.h + 0.5 * m.h * (xq[qy] + 1.0);
    z = cz * m.h + 0.5 * m.h * (xq[qz] + 1.0);
}

struct Tables1D {
    double xq[EFE_MAXNQ], wq[EFE_MAXNQ];
    double B1[EFE_MAXNQ * (EFE_MAXP + 1)], D1[EFE_MAXNQ * (EFE_MAXP + 1)];
};


inline Tables1D make_tables(const efe_ctx *ctx) {
    Tables1D T{};
    for (int q = 0; q < ctx->m.nq; ++q) {
        T.xq[q] = ctx->xq[q];
        T.wq[q] = ctx->wq[q];
        for (int a = 0; a <= ctx->m.p; ++a) {
            T.B1[q * ctx->m.np1 + a] = ctx->B1[q * ctx->m.np1 + a];
            T.D1[q * ctx->m.np1 + a] = ctx->D1[q * ctx->m.np1 + a];
        }
    }
    return T;
}

inline FuncParams make_fp(const efe_ctx *ctx) {
    FuncParams fp;
    fp.alpha = ctx->alpha;
    fp.r0 = ctx->r0;
    fp.t = ctx->t;
    fp.rc = ctx->rc;
    fp.rtrunc = ctx->rtrunc;
    fp.enrich = ctx->enrich ? 1 : 0;
    fp.nonlocal = ctx->nonlocal ? 1 : 0;
    return fp;
}


}  // namespace efe_dev

using namespace efe_dev;
