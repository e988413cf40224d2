// Register-resident small DFT codelets (radix 2, 3, 4, 5, 7, 8, 16, 32) in FP32.
//
// DIR = -1 is the forward kernel exp(-2 pi i / R), DIR = +1 the inverse.
// Every codelet maps a[0..R-1] (natural order) to its DFT (natural order),
// in place, unnormalised.  The composite radices 8 = 2 x 4, 16 = 4 x 4 and
// 32 = 4 x 8 are Cooley-Tukey splits with their inner twiddles as exact
// compile-time constants (values of cos/sin at multiples of pi/16, written to
// 20 digits).
#pragma once
#include <cuda_runtime.h>

namespace fft3d {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w)
{
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}
// a * (DIR * i)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a)
{
    return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// Multiply by the table twiddle W^m, where the table holds the forward
// (negative-sign) roots: DIR = +1 uses the conjugate.
template <int DIR>
__device__ __forceinline__ float2 twiddle(float2 a, float2 w_fwd)
{
    return DIR < 0 ? cmul(a, w_fwd) : cmulc(a, w_fwd);
}

// cos(2 pi m / 32) and sin(2 pi m / 32), m in [0, 32).
__device__ __forceinline__ constexpr float cos32(int m)
{
    constexpr float c[8] = {1.0f,
                            0.98078528040323044913f,
                            0.92387953251128675613f,
                            0.83146961230254523708f,
                            0.70710678118654752440f,
                            0.55557023301960222474f,
                            0.38268343236508977173f,
                            0.19509032201612826785f};
    // quarter-wave symmetry: cos on [0, 2 pi) from its first quarter
    const int q = (m & 31) >> 3, r = m & 7;
    return q == 0 ? c[r] : q == 1 ? (r == 0 ? 0.0f : -c[8 - r]) : q == 2 ? -c[r] : (r == 0 ? 0.0f : c[8 - r]);
}
__device__ __forceinline__ constexpr float sin32(int m) { return cos32(m + 24); }

// a * exp(DIR 2 pi i M / R) with M, R compile-time (R divides 32).
template <int R, int M, int DIR>
__device__ __forceinline__ float2 rot(float2 a)
{
    static_assert(32 % R == 0, "rotation grid is the 32nd roots of unity");
    constexpr int m32 = ((M % R) * (32 / R)) & 31;  // same angle on the 32-grid
    if constexpr (m32 == 0) {
        return a;
    } else if constexpr (m32 == 8) {
        return mul_i<DIR>(a);
    } else if constexpr (m32 == 16) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (m32 == 24) {
        return mul_i<-DIR>(a);
    } else {
        constexpr float c = cos32(m32);
        constexpr float s = DIR * sin32(m32);
        return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
    }
}

template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<1, DIR> {
    __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2* a)
    {
        float2 t = a[1];
        a[1] = csub(a[0], t);
        a[0] = cadd(a[0], t);
    }
};

template <int DIR>
struct Dft<3, DIR> {
    __device__ __forceinline__ static void run(float2* a)
    {
        constexpr float s3 = 0.86602540378443864676f;  // sin(2 pi / 3)
        float2 t1 = cadd(a[1], a[2]);
        float2 t2 = make_float2(fmaf(-0.5f, t1.x, a[0].x), fmaf(-0.5f, t1.y, a[0].y));
        float2 d = cscale(csub(a[1], a[2]), s3);
        float2 m = mul_i<DIR>(d);
        a[0] = cadd(a[0], t1);
        a[1] = cadd(t2, m);
        a[2] = csub(t2, m);
    }
};

template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2* a)
    {
        float2 s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
        float2 s13 = cadd(a[1], a[3]), d13 = mul_i<DIR>(csub(a[1], a[3]));
        a[0] = cadd(s02, s13);
        a[2] = csub(s02, s13);
        a[1] = cadd(d02, d13);
        a[3] = csub(d02, d13);
    }
};

template <int DIR>
struct Dft<5, DIR> {
    __device__ __forceinline__ static void run(float2* a)
    {
        constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
        constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
        constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
        constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
        float2 p14 = cadd(a[1], a[4]), m14 = csub(a[1], a[4]);
        float2 p23 = cadd(a[2], a[3]), m23 = csub(a[2], a[3]);
        float2 a0 = a[0];
        float2 r1 = make_float2(a0.x + c1 * p14.x + c2 * p23.x, a0.y + c1 * p14.y + c2 * p23.y);
        float2 r2 = make_float2(a0.x + c2 * p14.x + c1 * p23.x, a0.y + c2 * p14.y + c1 * p23.y);
        float2 i1 = mul_i<DIR>(make_float2(s1 * m14.x + s2 * m23.x, s1 * m14.y + s2 * m23.y));
        float2 i2 = mul_i<DIR>(make_float2(s2 * m14.x - s1 * m23.x, s2 * m14.y - s1 * m23.y));
        a[0] = cadd(a0, cadd(p14, p23));
        a[1] = cadd(r1, i1);
        a[4] = csub(r1, i1);
        a[2] = cadd(r2, i2);
        a[3] = csub(r2, i2);
    }
};

// 7 points: with t_j = a_j + a_{7-j}, d_j = a_j - a_{7-j} (j = 1, 2, 3),
//   X[m]   = a_0 + sum_j cos(2 pi j m / 7) t_j + DIR i sum_j sin(2 pi j m / 7) d_j,
//   X[7-m] = the same with the sine sum negated  (m = 1, 2, 3).
template <int DIR>
struct Dft<7, DIR> {
    __device__ __forceinline__ static void run(float2* a)
    {
        constexpr float c1 = 0.62348980185873353053f, c2 = -0.22252093395631440429f, c3 = -0.90096886790241912624f;
        constexpr float s1 = 0.78183148246802980871f, s2 = 0.97492791218182360702f, s3 = 0.43388373911755812048f;
        const float2 a0 = a[0];
        const float2 t1 = cadd(a[1], a[6]), d1 = csub(a[1], a[6]);
        const float2 t2 = cadd(a[2], a[5]), d2 = csub(a[2], a[5]);
        const float2 t3 = cadd(a[3], a[4]), d3 = csub(a[3], a[4]);
        // cos / sin of 2 pi (j m mod 7) / 7 for m = 1, 2, 3 and j = 1, 2, 3
        const float2 r1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x + c3 * t3.x, a0.y + c1 * t1.y + c2 * t2.y + c3 * t3.y);
        const float2 r2 = make_float2(a0.x + c2 * t1.x + c3 * t2.x + c1 * t3.x, a0.y + c2 * t1.y + c3 * t2.y + c1 * t3.y);
        const float2 r3 = make_float2(a0.x + c3 * t1.x + c1 * t2.x + c2 * t3.x, a0.y + c3 * t1.y + c1 * t2.y + c2 * t3.y);
        const float2 q1 = make_float2(s1 * d1.x + s2 * d2.x + s3 * d3.x, s1 * d1.y + s2 * d2.y + s3 * d3.y);
        const float2 q2 = make_float2(s2 * d1.x - s3 * d2.x - s1 * d3.x, s2 * d1.y - s3 * d2.y - s1 * d3.y);
        const float2 q3 = make_float2(s3 * d1.x - s1 * d2.x + s2 * d3.x, s3 * d1.y - s1 * d2.y + s2 * d3.y);
        const float2 i1 = mul_i<DIR>(q1), i2 = mul_i<DIR>(q2), i3 = mul_i<DIR>(q3);
        a[0] = cadd(a0, cadd(t1, cadd(t2, t3)));
        a[1] = cadd(r1, i1);
        a[6] = csub(r1, i1);
        a[2] = cadd(r2, i2);
        a[5] = csub(r2, i2);
        a[3] = cadd(r3, i3);
        a[4] = csub(r3, i3);
    }
};

// R = A * B split: n = na + A nb, k = kb + B ka.
//   Y[na][kb] = DFT_B over nb of a[na + A nb];  Y[na][kb] *= W_R^{na kb};
//   X[kb + B ka] = DFT_A over na of Y[na][kb].
template <int A, int B, int DIR>
struct DftSplit {
    template <int NA, int KB>
    __device__ __forceinline__ static void tw(float2 (&y)[A][B])
    {
        y[NA][KB] = rot<A * B, NA * KB, DIR>(y[NA][KB]);
        if constexpr (KB + 1 < B) tw<NA, KB + 1>(y);
        else if constexpr (NA + 1 < A) tw<NA + 1, 0>(y);
    }
    __device__ __forceinline__ static void run(float2* a)
    {
        float2 y[A][B];
#pragma unroll
        for (int na = 0; na < A; ++na) {
#pragma unroll
            for (int nb = 0; nb < B; ++nb) y[na][nb] = a[na + A * nb];
            Dft<B, DIR>::run(y[na]);
        }
        tw<1, 1>(y);
#pragma unroll
        for (int kb = 0; kb < B; ++kb) {
            float2 z[A];
#pragma unroll
            for (int na = 0; na < A; ++na) z[na] = y[na][kb];
            Dft<A, DIR>::run(z);
#pragma unroll
            for (int ka = 0; ka < A; ++ka) a[kb + B * ka] = z[ka];
        }
    }
};

template <int DIR>
struct Dft<8, DIR> {
    __device__ __forceinline__ static void run(float2* a) { DftSplit<2, 4, DIR>::run(a); }
};

template <int DIR>
struct Dft<16, DIR> {
    __device__ __forceinline__ static void run(float2* a) { DftSplit<4, 4, DIR>::run(a); }
};

template <int DIR>
struct Dft<32, DIR> {
    __device__ __forceinline__ static void run(float2* a) { DftSplit<4, 8, DIR>::run(a); }
};

}  // namespace fft3d
