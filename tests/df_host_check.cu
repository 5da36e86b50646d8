// Host driver for the double-float arithmetic of the integral kernels
// (paper_1905_01381_gb300/csrc/cq_df.cuh), used by test_df_host.py: reads
// lines "op a_hi a_lo b_hi b_lo c_hi c_lo" (FP32 values as hexadecimal bit
// patterns), applies the operation and prints the result's two words the
// same way.  op: 0 two_sum(a_hi, b_hi), 1 a + b, 2 a * b, 3 fma(a, b, c),
// 4 1/a, 5 sqrt(a).
#include <cstdio>
#include <cstring>
#include "cq_df.cuh"

using cq::df;

static float bits_to_float(unsigned u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

static unsigned float_to_bits(float f)
{
    unsigned u;
    std::memcpy(&u, &f, 4);
    return u;
}

int main()
{
    int op;
    unsigned w[6];
    while (std::scanf("%d %x %x %x %x %x %x", &op, &w[0], &w[1], &w[2], &w[3], &w[4], &w[5]) == 7) {
        const df a(bits_to_float(w[0]), bits_to_float(w[1]));
        const df b(bits_to_float(w[2]), bits_to_float(w[3]));
        const df c(bits_to_float(w[4]), bits_to_float(w[5]));
        df r(0.f, 0.f);
        switch (op) {
            case 0: r = cq::df_two_sum(a.hi, b.hi); break;
            case 1: r = a + b; break;
            case 2: r = a * b; break;
            case 3: r = cq::fma(a, b, c); break;
            case 4: r = cq::recip(a); break;
            case 5: r = cq::sqrt_df(a); break;
            default: return 2;
        }
        std::printf("%08x %08x\n", float_to_bits(r.hi), float_to_bits(r.lo));
    }
    return 0;
}
