// Division of cell indices by invariant grid extents without a hardware divide.
//
// Granlund & Montgomery, "Division by invariant integers using multiplication" (PLDI 1994),
// Theorem 4.2: for N-bit numerators and a divisor d >= 1, with l = ceil(log2 d),
// s = N + l and m = ceil(2^s / d), floor(n / d) = floor(n m / 2^s) for every 0 <= n < 2^N.
// Cell indices are below 2^31 (N = 31), so m <= 2^32 and n m < 2^63: one 64-bit multiply and a
// shift replace the ~70-instruction 64-bit integer division of the stencil kernels' index
// arithmetic.
#pragma once

#ifdef __CUDACC__
#define RHI_HD __host__ __device__
#else
#define RHI_HD
#endif

namespace rhi {

struct FastDiv {
    unsigned long long m;   // ceil(2^s / d)
    unsigned s;             // 31 + ceil(log2 d)
    unsigned d;
};

inline FastDiv make_fastdiv(unsigned d) {
    unsigned l = 0;
    while (l < 32 && (1ULL << l) < (unsigned long long)d) ++l;
    FastDiv f;
    f.d = d;
    f.s = 31 + l;
    f.m = ((1ULL << f.s) + d - 1) / d;
    return f;
}

// n / f.d for 0 <= n < 2^31
RHI_HD inline unsigned fdiv(unsigned n, const FastDiv& f) {
    return (unsigned)(((unsigned long long)n * f.m) >> f.s);
}

}  // namespace rhi
