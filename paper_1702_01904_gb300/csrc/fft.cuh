// fft.cuh -- register-resident DFTs and a two-level block FFT for sm_103a.
//
// Convention (as in the rest of the library): forward X[k] = sum_n x[n] exp(-2 pi i n k / N),
// inverse without normalisation (exp(+2 pi i n k / N)); callers fold 1/N where needed.
//
// Structure.  A length-N transform is split as N = N1 * N2 (four-step / Stockham form):
//   X[k1 + N1 k2] = sum_{n2} W_N2^{n2 k2} * ( W_N^{n2 k1} * sum_{n1} x[N2 n1 + n2] W_N1^{n1 k1} ).
// T = N / E threads cooperate on one transform, each holding E = max(N1, N2) elements in
// registers.  Stage 1 is a radix-N1 DFT in registers, then the inter-stage twiddle, one
// exchange through shared memory, and stage 2 is a radix-N2 DFT in registers.  Register DFTs of
// size 16..64 are themselves split recursively at compile time with twiddles held in kernel
// parameter space (constant bank), so every index below is a compile-time constant.
//
// Register layouts (thread t, J = E/N1, I = E/N2):
//   input : reg n1*J + j  holds element  N2*n1 + t + T*j
//   output: reg k2*I + i  holds element  t + T*i + N1*k2
// A forward transform with split (A, B) leaves its output in exactly the input layout of an
// inverse transform with split (B, A), and vice versa, so FFT -> pointwise -> IFFT chains need no
// data movement between transforms.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "params.h"  // Tw64: W_64^j = exp(-2 pi i j / 64), computed on the host in double

namespace prism {

// Complex additions issue as one packed FP32x2 instruction (sm_100 family): the same IEEE
// round-to-nearest result per component as two scalar additions, in half the issue slots.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }

// multiply by W_4 (forward: -i, inverse: +i)
template <bool INV>
__device__ __forceinline__ float2 rot4(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// multiply by W_64^J (forward) or W_64^-J (inverse); J is a compile-time constant.
template <int J, bool INV>
__device__ __forceinline__ float2 twiddle64(float2 a, const Tw64 &tw) {
    constexpr int j = J & 63;
    constexpr float r = 0.70710678118654752440f;  // sqrt(1/2)
    if constexpr (j == 0) {
        return a;
    } else if constexpr (j == 16) {
        return rot4<INV>(a);
    } else if constexpr (j == 32) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (j == 48) {
        return rot4<!INV>(a);
    } else if constexpr (j == 8) {  // (1 - i)/sqrt2 forward
        return INV ? make_float2((a.x - a.y) * r, (a.x + a.y) * r) : make_float2((a.x + a.y) * r, (a.y - a.x) * r);
    } else if constexpr (j == 24) {  // (-1 - i)/sqrt2 forward
        return INV ? make_float2(-(a.x + a.y) * r, (a.x - a.y) * r) : make_float2((a.y - a.x) * r, -(a.x + a.y) * r);
    } else if constexpr (j == 40) {  // (-1 + i)/sqrt2 forward
        return INV ? make_float2((a.y - a.x) * r, -(a.x + a.y) * r) : make_float2(-(a.x + a.y) * r, (a.x - a.y) * r);
    } else if constexpr (j == 56) {  // (1 + i)/sqrt2 forward
        return INV ? make_float2((a.x + a.y) * r, (a.y - a.x) * r) : make_float2((a.x - a.y) * r, (a.x + a.y) * r);
    } else {
        return INV ? cmulc(a, tw.w[j]) : cmul(a, tw.w[j]);
    }
}

// fn(std::integral_constant<int, r>) for r = 0 ... N-1, unrolled at compile time (lets the body
// branch on compile-time properties of the register index)
template <class Fn, int... Is>
__device__ __forceinline__ void static_for_impl(Fn &fn, std::integer_sequence<int, Is...>) {
    (fn(std::integral_constant<int, Is>{}), ...);
}
template <int N, class Fn>
__device__ __forceinline__ void static_for(Fn fn) {
    static_for_impl(fn, std::make_integer_sequence<int, N>{});
}
// Tangent form of W_64^J (INV: of its conjugate), for butterflies that take the twiddle's scale
// into a packed FMA: W y = s u with
//   |cos| >= |sin| ((J mod 32) <= 8 or >= 24): s = cos, k = tan, u = (y.x - k y.y, y.y + k y.x)
//   otherwise:                                   s = sin, k = cot, u = (k y.x - y.y, k y.y + y.x)
// (the conjugate flips k, and in the cot form also s).  Multiples of 16 are free rotations and are
// not put in this form.
template <int J>
struct TanForm {
    static constexpr int j = J & 63;
    static constexpr bool tan = (j & 31) <= 8 || (j & 31) >= 24;
    static constexpr bool rotation = (j & 15) == 0;  // 1, -i, -1, +i: no multiply
};

template <int J, bool INV>
__device__ __forceinline__ float2 tan_u(float2 y, const Tw64 &tw) {
    constexpr int j = TanForm<J>::j;
    const float k = tw.tk[j];
    if constexpr (TanForm<J>::tan) {
        return INV ? make_float2(fmaf(k, y.y, y.x), fmaf(-k, y.x, y.y)) : make_float2(fmaf(-k, y.y, y.x), fmaf(k, y.x, y.y));
    } else {
        return INV ? make_float2(fmaf(-k, y.x, -y.y), fmaf(-k, y.y, y.x)) : make_float2(fmaf(k, y.x, -y.y), fmaf(k, y.y, y.x));
    }
}

template <int J, bool INV>
__device__ __forceinline__ float2 tan_s(const Tw64 &tw) {
    const float2 s = tw.sc[TanForm<J>::j];
    return (!TanForm<J>::tan && INV) ? make_float2(-s.x, -s.y) : s;
}

__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }

// Known zeros.  The codelets below take a compile-time mask Z of inputs that are exactly zero in
// every thread (bit i: element i S), e.g. the frequencies the anti-aliasing aperture removed, and
// leave out the arithmetic on them (the compiler may not drop x + 0 itself: -0 + 0 is +0).
__host__ __device__ constexpr bool zbit(unsigned long long z, int i) { return (z >> i) & 1ull; }

template <bool ZA, bool ZB>
__device__ __forceinline__ float2 zadd(float2 a, float2 b) {
    if constexpr (ZA && ZB) return make_float2(0.f, 0.f);
    else if constexpr (ZB) return a;
    else if constexpr (ZA) return b;
    else return cadd(a, b);
}
template <bool ZA, bool ZB>
__device__ __forceinline__ float2 zsub(float2 a, float2 b) {
    if constexpr (ZA && ZB) return make_float2(0.f, 0.f);
    else if constexpr (ZB) return a;
    else if constexpr (ZA) return cneg(b);
    else return csub(a, b);
}

// One input of a twiddled DFT-4: exactly zero, a plain value (twiddle 1 or a free rotation), or
// s u (a tangent-form twiddle, see tan_u / tan_s).
enum { TERM_ZERO = 0, TERM_PLAIN = 1, TERM_SCALED = 2 };
template <int J, bool Z, bool INV>
struct Term {
    static constexpr int kind = Z ? TERM_ZERO : TanForm<J>::rotation ? TERM_PLAIN : TERM_SCALED;
    float2 v, s;  // PLAIN: v; SCALED: u in v, scale in s
    __device__ __forceinline__ Term(float2 y, const Tw64 &tw) {
        if constexpr (kind == TERM_PLAIN) {
            v = twiddle64<J, INV>(y, tw);
        } else if constexpr (kind == TERM_SCALED) {
            v = tan_u<J, INV>(y, tw);
            s = tan_s<J, INV>(tw);
        }
    }
};
// a + b and a - b of two terms (plain results); a SCALED a and b share the product s_a u_a
template <class TA, class TB>
__device__ __forceinline__ void term_sum_diff(const TA &a, const TB &b, float2 &sum, float2 &diff) {
    constexpr int ka = TA::kind, kb = TB::kind;
    if constexpr (ka == TERM_ZERO && kb == TERM_ZERO) {
        sum = diff = make_float2(0.f, 0.f);
    } else if constexpr (kb == TERM_ZERO) {
        sum = diff = ka == TERM_PLAIN ? a.v : __fmul2_rn(a.s, a.v);
    } else if constexpr (ka == TERM_ZERO) {
        sum = kb == TERM_PLAIN ? b.v : __fmul2_rn(b.s, b.v);
        diff = kb == TERM_PLAIN ? cneg(b.v) : __fmul2_rn(cneg(b.s), b.v);
    } else if constexpr (ka == TERM_PLAIN && kb == TERM_PLAIN) {
        sum = cadd(a.v, b.v);
        diff = csub(a.v, b.v);
    } else if constexpr (ka == TERM_PLAIN) {
        sum = __ffma2_rn(b.s, b.v, a.v);
        diff = __ffma2_rn(cneg(b.s), b.v, a.v);
    } else if constexpr (kb == TERM_PLAIN) {
        sum = __ffma2_rn(a.s, a.v, b.v);
        diff = __ffma2_rn(a.s, a.v, cneg(b.v));
    } else {
        const float2 p = __fmul2_rn(a.s, a.v);
        sum = __ffma2_rn(b.s, b.v, p);
        diff = __ffma2_rn(cneg(b.s), b.v, p);
    }
}

// DFT-4 of (x[0], W^J1 x[S], W^J2 x[2S], W^J3 x[3S]) (W = W_64, conjugated for INV), natural order
// in and out, with every twiddle in tangent form: its scale enters the butterfly's packed FMA, so a
// twiddled input costs 2 FP32 lane operations on top of the plain DFT-4 instead of 4.  Z: known
// zero inputs.
template <int J1, int J2, int J3, int S, bool INV, unsigned long long Z = 0>
struct Dft4Tw {
    __device__ __forceinline__ static void run(float2 *x, const Tw64 &tw) {
        const Term<0, zbit(Z, 0), INV> t0(x[0], tw);
        const Term<J1, zbit(Z, 1), INV> t1(x[S], tw);
        const Term<J2, zbit(Z, 2), INV> t2(x[2 * S], tw);
        const Term<J3, zbit(Z, 3), INV> t3(x[3 * S], tw);
        float2 A, B, C, D;  // x0 +- W^J2 x2, W^J1 x1 +- W^J3 x3
        term_sum_diff(t0, t2, A, B);
        term_sum_diff(t1, t3, C, D);
        constexpr bool zac = zbit(Z, 0) && zbit(Z, 2), zc = zbit(Z, 1) && zbit(Z, 3);
        const float2 rd = rot4<INV>(D);
        x[0] = zadd<zac, zc>(A, C);
        x[2 * S] = zsub<zac, zc>(A, C);
        x[S] = zadd<zac, zc>(B, rd);
        x[3 * S] = zsub<zac, zc>(B, rd);
    }
};

// In-place DFT of R elements x[0], x[S], ..., x[(R-1)S]; natural order in and out.  Z: inputs known
// to be exactly zero (bit i: element i S).  V: split variant of the 32- and 64-point codelets
// (DftSplit); the 1- to 8-point codelets have one form.
template <int R, int S, bool INV, unsigned long long Z = 0, int V = 0>
struct Dft;

template <int S, bool INV, unsigned long long Z, int V>
struct Dft<1, S, INV, Z, V> {
    __device__ __forceinline__ static void run(float2 *, const Tw64 &) {}
};

template <int S, bool INV, unsigned long long Z, int V>
struct Dft<2, S, INV, Z, V> {
    __device__ __forceinline__ static void run(float2 *x, const Tw64 &) {
        float2 a = x[0], b = x[S];
        x[0] = zadd<zbit(Z, 0), zbit(Z, 1)>(a, b);
        x[S] = zsub<zbit(Z, 0), zbit(Z, 1)>(a, b);
    }
};

template <int S, bool INV, unsigned long long Z, int V>
struct Dft<4, S, INV, Z, V> {
    __device__ __forceinline__ static void run(float2 *x, const Tw64 &) {
        constexpr bool z0 = zbit(Z, 0), z1 = zbit(Z, 1), z2 = zbit(Z, 2), z3 = zbit(Z, 3);
        float2 t0 = zadd<z0, z2>(x[0], x[2 * S]);
        float2 t1 = zsub<z0, z2>(x[0], x[2 * S]);
        float2 t2 = zadd<z1, z3>(x[S], x[3 * S]);
        float2 t3 = rot4<INV>(zsub<z1, z3>(x[S], x[3 * S]));
        x[0] = zadd<z0 && z2, z1 && z3>(t0, t2);
        x[2 * S] = zsub<z0 && z2, z1 && z3>(t0, t2);
        x[S] = zadd<z0 && z2, z1 && z3>(t1, t3);
        x[3 * S] = zsub<z0 && z2, z1 && z3>(t1, t3);
    }
};

template <int S, bool INV, unsigned long long Z, int V>
struct Dft<8, S, INV, Z, V> {
    __device__ __forceinline__ static void run(float2 *x, const Tw64 &tw) {
        // decimation in frequency: b_k = a_k + a_{k+4} (even outputs), c_k = (a_k - a_{k+4}) W8^k (odd)
        float2 b[4], c[4];
        static_for<4>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            b[k] = zadd<zbit(Z, k), zbit(Z, k + 4)>(x[k * S], x[(k + 4) * S]);
            c[k] = zsub<zbit(Z, k), zbit(Z, k + 4)>(x[k * S], x[(k + 4) * S]);
        });
        constexpr unsigned long long ZH = (Z & (Z >> 4)) & 15ull;  // b_k, c_k zero when both inputs are
        Dft<4, 1, INV, ZH>::run(b, tw);
        Dft4Tw<8, 16, 24, 1, INV, ZH>::run(c, tw);  // c_k W_8^k, then the DFT-4
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            x[(2 * m) * S] = b[m];
            x[(2 * m + 1) * S] = c[m];
        }
    }
};

// Split R = R1 x R2 of the larger register DFTs (stage 1: R2 DFTs of R1 points, stage 2: R1 DFTs of
// R2 points).  Variant 0: R1 = 4 for 16, 8 for 32 and 64 (16 = 4 x 4, 32 = 8 x 4 with the radix-4
// second stage taking its twiddles in tangent form, 64 = 8 x 8).  Variant 1: a radix-4 first stage
// (32 = 4 x 8, 64 = 4 x 16), whose DFT-4s are cheap where the inputs are known zeros (the band-
// limited inputs of the passes) but whose second stage multiplies its twiddles separately.  Both
// compute the same DFT; they round differently.
template <int R, int V = 0>
struct DftSplit {
    static constexpr int R1 = (R != 16 && R != 32 && R != 64) ? 0 : (R == 16 || V == 1) ? 4 : 8;
    static constexpr int R2 = R1 ? R / R1 : 0;
};

template <int R1, int R2, int S, bool INV, int N2>
struct DftTw {
    // multiply element (R2*k1 + n2) by W_R^{n2 k1}, for all n2 < R2, k1 < R1
    template <int K>
    __device__ __forceinline__ static void go(float2 *x, const Tw64 &tw) {
        if constexpr (K < R1 * R2) {
            constexpr int k1 = K / R2, n2 = K % R2;
            x[(R2 * k1 + n2) * S] = twiddle64<(n2 * k1 * (64 / (R1 * R2))) & 63, INV>(x[(R2 * k1 + n2) * S], tw);
            go<K + 1>(x, tw);
        }
    }
};

// bits n1 < R1 of a mask over elements R2 n1 + n2 (the inputs of stage-1 sub-DFT n2)
template <int R1, int R2>
__host__ __device__ constexpr unsigned long long sub_mask(unsigned long long z, int n2) {
    unsigned long long m = 0;
    for (int n1 = 0; n1 < R1; ++n1)
        if (zbit(z, R2 * n1 + n2)) m |= 1ull << n1;
    return m;
}
// stage-2 inputs known zero: those of stage-1 sub-DFTs whose inputs were all zero
template <int R1, int R2>
__host__ __device__ constexpr unsigned long long stage2_mask(unsigned long long z) {
    unsigned long long m = 0;
    for (int n2 = 0; n2 < R2; ++n2)
        if (sub_mask<R1, R2>(z, n2) == (R1 >= 64 ? ~0ull : ((1ull << R1) - 1))) m |= 1ull << n2;
    return m;
}

template <int R, int S, bool INV, unsigned long long Z, int V>
struct Dft {
    static constexpr int R1 = DftSplit<R, V>::R1;
    static constexpr int R2 = DftSplit<R, V>::R2;
    static_assert(R1 > 0, "unsupported register DFT size");
    __device__ __forceinline__ static void run(float2 *x, const Tw64 &tw) {
        // stage 1: DFT over n1 of elements (R2 n1 + n2) for each n2
        static_for<R2>([&](auto nc) {
            constexpr int n2 = decltype(nc)::value;
            Dft<R1, R2 * S, INV, sub_mask<R1, R2>(Z, n2), V>::run(x + n2 * S, tw);
        });
        // stage 2: DFT over n2 of elements (R2 k1 + n2) times W_R^{n2 k1}, for each k1 -> X[k1 + R1 k2]
        // at (R2 k1 + k2); radix 4 with the twiddles in the butterflies, else twiddles then DFTs
        constexpr unsigned long long Z2 = stage2_mask<R1, R2>(Z);
        if constexpr (R2 == 4) {
            static_for<R1>([&](auto kc) {
                constexpr int k1 = decltype(kc)::value, jj = k1 * (64 / R);
                Dft4Tw<jj, 2 * jj, 3 * jj, S, INV, Z2>::run(x + R2 * k1 * S, tw);
            });
        } else {
            static_assert(Z2 == 0, "known-zero stage-2 inputs need the radix-4 stage");
            DftTw<R1, R2, S, INV, R2>::template go<0>(x, tw);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) Dft<R2, S, INV, 0, V>::run(x + R2 * k1 * S, tw);
        }
        float2 tmp[R];
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) tmp[k1 + R1 * k2] = x[(R2 * k1 + k2) * S];
#pragma unroll
        for (int k = 0; k < R; ++k) x[k * S] = tmp[k];
    }
};

// ----------------------------------------------------------------------------------------
// Split of each supported length into (N1, N2) for the forward transform; the inverse uses
// (N2, N1) so that forward-out == inverse-in layouts.
template <int N>
struct FftShape {
    static constexpr int N1 = (N == 8) ? 4 : (N == 16) ? 4 : (N == 32) ? 8 : (N == 64) ? 8 : (N == 128) ? 16
                            : (N == 256) ? 16 : (N == 512) ? 32 : (N == 1024) ? 32 : (N == 2048) ? 64 : 0;
    static constexpr int N2 = N1 ? N / N1 : 0;
    static constexpr int E = N1 > N2 ? N1 : N2;
    static constexpr int T = N / E;
    static_assert(N1 > 0, "unsupported FFT length");
};

// Where BlockFft::run finds its inter-stage twiddle table and in which order it reads it
enum { TW_SMEM = 0, TW_GLOBAL = 1, TW_SMEM_SEQ = 2 };

// A no-op in place of BlockFft::run's hook
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// Two-level transform of length N = N1*N2 over T threads.  `stw` is the inter-stage twiddle
// table laid out [k1][n2] = W_N^{n2 k1} (forward sign; the inverse conjugates it); kernels keep
// it in shared memory (lanes read consecutive n2: conflict-free).  `Ex` is the exchange:
// write(k1, n2, v), read(k1, n2), sync().
// V: split variant of the register DFTs (DftSplit)
template <int N1, int N2, bool INV, int V = 0>
struct BlockFft {
    static constexpr int SPLIT1 = N1, SPLIT2 = N2;  // first-stage, second-stage DFT lengths
    static constexpr int N = N1 * N2;
    static constexpr int E = N1 > N2 ? N1 : N2;
    static constexpr int T = N / E;
    static constexpr int J = E / N1;
    static constexpr int I = E / N2;

    // GTW: where the twiddle table is and how it is read: TW_SMEM (shared memory, every twiddle
    // loaded before the first exchange store), TW_GLOBAL (global memory through the read-only path,
    // each twiddle loaded, applied and stored in turn, which keeps register pressure at the level
    // of one element) or TW_SMEM_SEQ (shared memory, read in that interleaved order)
    // ZIN: input registers known to be exactly zero in every thread (bit r: register r)
    // LEAD: synchronise before the exchange is written (off where the caller has already ordered
    // every earlier access of the buffer before this call's writes)
    // hook(): called by every thread right after the barrier that follows the exchange writes
    template <class Ex, int GTW = TW_SMEM, unsigned long long ZIN = 0, bool LEAD = true, class Hook = NoHook>
    __device__ __forceinline__ static void run(float2 (&x)[E], int t, const float2 *__restrict__ stw,
                                               const Tw64 &tw, Ex &ex, Hook hook = Hook{}) {
        static_for<J>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            Dft<N1, J, INV, sub_mask<N1, J>(ZIN, j), V>::run(x + j, tw);
        });
        if constexpr (GTW == TW_SMEM) {
            // shared-memory table: all twiddle loads before any exchange store (the table and the
            // exchange share the address space, and this order lets the loads issue back to back)
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int n2 = t + T * j;
#pragma unroll
                for (int k1 = 1; k1 < N1; ++k1) {
                    const float2 w = stw[k1 * N2 + n2];
                    x[k1 * J + j] = INV ? cmulc(x[k1 * J + j], w) : cmul(x[k1 * J + j], w);
                }
            }
            if constexpr (LEAD) ex.sync();  // previous readers of the exchange are done
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int n2 = t + T * j;
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) ex.write(k1, n2, x[k1 * J + j]);
            }
        } else {
            // interleave load, multiply and store (TW_GLOBAL: read-only path, L1-resident)
            if constexpr (LEAD) ex.sync();
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int n2 = t + T * j;
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) {
                    float2 v = x[k1 * J + j];
                    if (k1 != 0) {
                        const float2 w = GTW == TW_GLOBAL ? __ldg(stw + k1 * N2 + n2) : stw[k1 * N2 + n2];
                        v = INV ? cmulc(v, w) : cmul(v, w);
                    }
                    ex.write(k1, n2, v);
                }
            }
        }
        ex.sync();
        hook();
#pragma unroll
        for (int i = 0; i < I; ++i) {
            const int k1 = t + T * i;
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) x[n2 * I + i] = ex.read(k1, n2);
        }
#pragma unroll
        for (int i = 0; i < I; ++i) Dft<N2, I, INV, 0, V>::run(x + i, tw);
    }

    // element index held in register r (input / output layouts)
    __host__ __device__ __forceinline__ static constexpr int in_elem(int r, int t) { return N2 * (r / J) + t + T * (r % J); }
    __host__ __device__ __forceinline__ static constexpr int out_elem(int r, int t) { return t + T * (r % I) + N1 * (r / I); }
};

// Band classes of the registers of a transform of length N for the band |k| < N/4 (FFT order):
// BAND_OUT if register r holds an element outside the band in every thread, BAND_IN if inside in
// every thread, BAND_MIXED otherwise.  With the band known at compile time, a register that is
// BAND_OUT in the input is a literal zero and one that is BAND_OUT in the output is never used, so
// the compiler removes their arithmetic from the first and the last register DFT.
enum { BAND_IN = 0, BAND_OUT = 1, BAND_MIXED = 2 };

template <class F, int N>
struct BandClass {
    __host__ __device__ static constexpr bool in_band(int e) { return e < N / 4 || e > N - N / 4; }
    __host__ __device__ static constexpr int of(int r, bool input) {
        bool any_in = false, any_out = false;
        for (int t = 0; t < F::T; ++t) {
            const int e = input ? F::in_elem(r, t) : F::out_elem(r, t);
            (in_band(e) ? any_in : any_out) = true;
        }
        return any_in && any_out ? BAND_MIXED : any_in ? BAND_IN : BAND_OUT;
    }
};

// registers that hold a band-outside element in every thread (input or output layout): known zeros
template <class F, int N>
__host__ __device__ constexpr unsigned long long band_zero_mask(bool input) {
    unsigned long long m = 0;
    for (int r = 0; r < F::E; ++r)
        if (BandClass<F, N>::of(r, input) == BAND_OUT) m |= 1ull << r;
    return m;
}

template <int N, int V = 0>
using FwdFft = BlockFft<FftShape<N>::N1, FftShape<N>::N2, false, V>;
template <int N, int V = 0>
using InvFft = BlockFft<FftShape<N>::N2, FftShape<N>::N1, true, V>;

// Exchange for transforms held by T consecutive lanes of one warp (T <= 32); each transform
// owns N1*(N2+1) float2 of shared memory (the +1 pad keeps stage-2 reads at two wavefronts).
template <int N1, int N2, int T>
struct WarpExchange {
    float2 *buf;
    __device__ __forceinline__ void write(int k1, int n2, float2 v) { buf[k1 * (N2 + 1) + n2] = v; }
    __device__ __forceinline__ float2 read(int k1, int n2) const { return buf[k1 * (N2 + 1) + n2]; }
    __device__ __forceinline__ void sync() { __syncwarp(); }
    static constexpr int kFloats2 = N1 * (N2 + 1);
};

// Exchange for W interleaved columns handled by a whole CTA: layout [k1][n2][c], each k1 block
// padded by W float2 so that the thread groups of a warp reading consecutive k1 in stage 2 fall on
// different banks.  Size: N1 * (N2 + 1) * W float2.
template <int N1, int N2, int W>
struct ColExchange {
    float2 *buf;
    int c;
    __device__ __forceinline__ void write(int k1, int n2, float2 v) { buf[(k1 * (N2 + 1) + n2) * W + c] = v; }
    __device__ __forceinline__ float2 read(int k1, int n2) const { return buf[(k1 * (N2 + 1) + n2) * W + c]; }
    __device__ __forceinline__ void sync() { __syncthreads(); }
    static constexpr int kFloats2 = N1 * (N2 + 1) * W;
};

// float2 count of a column exchange serving both the forward and the inverse split of length N
template <int N, int W>
struct ColExSize {
    static constexpr int a = FftShape<N>::N1, b = FftShape<N>::N2;
    static constexpr int value = (a * (b + 1) > b * (a + 1) ? a * (b + 1) : b * (a + 1)) * W;
};

}  // namespace prism
