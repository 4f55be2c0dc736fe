// Checks the integer-operation conversion and split of efe_convert.cuh
// against the hardware conversion and FP64 over hashed bit patterns, and the
// double-single product difference against FP64: every binary64 exponent
// range that maps onto binary32 normals, subnormals, overflow and zero,
// exact ties, and NaN / inf.  Prints the mismatch counts; exit status 0.
#include <cmath>
#include <cstdio>
#include "efe_convert.cuh"

__device__ unsigned long long mix(unsigned long long h) {
    h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29; h *= 0x94D049BB133111EBull; h ^= h >> 32;
    return h;
}

__global__ void k_check(long long n, unsigned long long *bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long h = mix((unsigned long long)i * 0x9E3779B97F4A7C15ull + 1);
        unsigned long long b = h;
        switch (i & 7) {
            case 0: case 1: case 2: {   // exponents around the binary32 range
                const int e = 1023 - 160 + (int)((h >> 52) % 330);
                b = (h & 0x800fffffffffffffull) | ((unsigned long long)e << 52);
                break;
            }
            case 3: {                   // exact ties and their neighbours
                const int e = 1023 - 155 + (int)((h >> 52) % 290);
                b = (h & 0x800fffffe0000000ull) | ((unsigned long long)e << 52) | 0x10000000ull;
                b += (unsigned long long)((long long)((h >> 8) % 3) - 1);
                break;
            }
            case 4: b = (h & 0x800fffffffffffffull) | (0x7ffull << 52); break;   // inf / NaN
            default: break;             // anything
        }
        const double x = __longlong_as_double((long long)b);
        const float got = f64_to_f32_rn(x), ref = __double2float_rn(x);
        if (x != x) {
            if (got == got) atomicAdd(&bad[0], 1ull);
        } else if (__float_as_uint(got) != __float_as_uint(ref)) {
            atomicAdd(&bad[0], 1ull);
        }
        // the split: hi is the hardware's rounding, and hi + lo reproduces x to 2^-45
        // relative where hi and lo are binary32 normals
        if (x == x) {
            float hi, lo;
            f64_split(x, hi, lo);
            const bool in = fabs(x) >= 0x1p-100 && fabs(x) < 0x1p120;
            if (__float_as_uint(hi) != __float_as_uint(ref) ||
                (in && !(fabs(x - ((double)hi + (double)lo)) < 0x1p-45 * fabs(x))))
                atomicAdd(&bad[1], 1ull);
        }
        // the double-single difference a b - c d against FP64, on operands of one scale
        // with cancellation down to 2^-20 of the products
        {
            const double a = 1.0 + (double)(h & 0xffffff) * 0x1p-24, bq = 0.5 + (double)((h >> 24) & 0xffffff) * 0x1p-25;
            const double c = 1.0 + (double)((h >> 48) & 0xffff) * 0x1p-16;
            const double d = (a * bq / c) * (1.0 + ldexp((double)((h >> 8) & 0xffff) - 32768.0, -35));
            float ah, al, bh, bl, ch, cl, dh, dl;
            f64_split(a, ah, al);
            f64_split(bq, bh, bl);
            f64_split(c, ch, cl);
            f64_split(d, dh, dl);
            const float got2 = ds_mul_sub(ah, al, bh, bl, ch, cl, dh, dl);
            const double exact = fma(a, bq, -c * d);   // cancels to <= 2^-20 |a b|: FP64 error ~2^-53 |a b|
            const double tol = ldexp(fabs((double)got2), -23) + 0x1p-43 * (fabs(a * bq) + fabs(c * d));
            if (fabs((double)got2 - exact) > tol) atomicAdd(&bad[2], 1ull);
        }
    }
}

int main() {
    const long long n = 1LL << 28;
    unsigned long long *bad = nullptr, hb[3] = {0, 0, 0};
    if (cudaMalloc(&bad, sizeof(hb)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, sizeof(hb));
    k_check<<<4096, 256>>>(n, bad);
    if (cudaMemcpy(hb, bad, sizeof(hb), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    printf("checked %lld f64_to_f32_rn %llu f64_split %llu ds_mul_sub %llu\n", n, hb[0], hb[1], hb[2]);
    return 0;
}
