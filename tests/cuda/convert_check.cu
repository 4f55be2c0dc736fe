// Checks the integer-operation conversion of efe_convert.cuh against the
// hardware conversion over hashed bit patterns: every binary64 exponent
// range that maps onto binary32 normals, subnormals, overflow and zero,
// exact ties, and NaN / inf.  Prints the mismatch counts; exit status 0.
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
    }
}

int main() {
    const long long n = 1LL << 28;
    unsigned long long *bad = nullptr, hb[1] = {0};
    if (cudaMalloc(&bad, sizeof(hb)) != cudaSuccess) return 2;
    cudaMemset(bad, 0, sizeof(hb));
    k_check<<<4096, 256>>>(n, bad);
    if (cudaMemcpy(hb, bad, sizeof(hb), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    printf("checked %lld f64_to_f32_rn %llu\n", n, hb[0]);
    return 0;
}
