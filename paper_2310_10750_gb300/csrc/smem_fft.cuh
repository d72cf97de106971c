// Periodic disc sums of a small lattice by FFT in shared memory, FP32 or FP64.
//
// On the periodic lattice the nodal quadrature of Section 2, S_i = sum_{z in D} w_z u_{i+z}, is a
// circular convolution, S = IFFT2(FFT2(u) K^), where K^ is the transform of the disc weights.
// The disc and the radial weights are even in dx and in dy, so K^ is real (formed on the host,
// divided by n^2 for the two unnormalised inverse transforms).  One CTA computes the sums of one
// sample:
//
//   row pass      each pair of rows (2p, 2p + 1) as one complex row z = u_2p + i u_2p+1, its
//                 forward transform Z, split into the two real rows' half spectra
//                 A_k = (Z_k + conj Z_{n-k}) / 2 and B_k = (Z_k - conj Z_{n-k}) / 2i, k <= n/2;
//   column pass   each half-spectrum column kx: forward transform over ky, product with
//                 K^(ky, kx), inverse transform;
//   row pass      the pair's rows of the product combined into Z_k = A_k + i B_k (the upper half
//                 by Hermitian symmetry), whose inverse transform is S_2p + i S_2p+1.
//
// The half spectrum [ky][kx] (n x (n/2 + 1) complex values) stays in shared memory; each warp
// transforms one sequence at a time in two buffers of n complex values of its own.  The 1-D
// transform is a mixed-radix Stockham FFT (self-sorting, natural order in and out) with radices
// 4, 2 and the odd primes up to 11, so it serves every even n whose odd part factors into those
// primes (the paper's meshes 64, 88 = 8 x 11 and 128 among them).  Stage s with radix p after
// L = p_1 ... p_{s-1} (r = n / (L p)) maps the partial transforms y[k0][m] of length L of the
// r p interleaved subsequences to those of length L p of r subsequences:
//     y'[k0 + L k1][m] = sum_q W_p^(q k1) W_{Lp}^(q k0) y[k0][m + q r],
// stored y[k][m] at k r_s + m for the stage's r_s subsequences; W_{Lp} = W_n^r, so one table
// of W_n^j = exp(-2 pi i j / n), j < n, gives every twiddle (conjugated for the inverse).
#pragma once

#include <cuda_runtime.h>

namespace mfmc {

constexpr int kFftMaxStages = 12;
constexpr int kFftMaxN = 128;  // the largest lattice whose half spectrum the CTA holds

// Radix plan of an n-point transform (host-built).
struct FftPlan {
    int n = 0;
    int stages = 0;
    int radix[kFftMaxStages] = {};
};

// Radices of n: the odd primes 11 .. 3 first (the first stage has no twiddle products, and an
// odd radix has the most), then 4 while 4 divides it, then 2.  False when another prime factor
// is left (the transform does not serve that n).
inline bool fft_plan(int n, FftPlan *p) {
    p->n = n;
    p->stages = 0;
    int m = n;
    static const int rs[] = {11, 7, 5, 3, 4, 2};
    for (int r : rs)
        while (m % r == 0 && p->stages < kFftMaxStages) {
            p->radix[p->stages++] = r;
            m /= r;
        }
    return m == 1 && n >= 2;
}

template <typename T>
struct FftCx;
template <>
struct FftCx<float> {
    using t = float2;
};
template <>
struct FftCx<double> {
    using t = double2;
};

template <typename C>
__device__ __forceinline__ C fcx(decltype(C().x) a, decltype(C().x) b) {
    C c;
    c.x = a;
    c.y = b;
    return c;
}
template <typename C>
__device__ __forceinline__ C fadd(C a, C b) {
    return fcx<C>(a.x + b.x, a.y + b.y);
}
template <typename C>
__device__ __forceinline__ C fsub(C a, C b) {
    return fcx<C>(a.x - b.x, a.y - b.y);
}
// a * w, or a * conj(w) for the inverse transform
template <bool INV, typename C>
__device__ __forceinline__ C fmulw(C a, C w) {
    return INV ? fcx<C>(a.x * w.x + a.y * w.y, a.y * w.x - a.x * w.y)
               : fcx<C>(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
// -i a (forward) or +i a (inverse): the factor W_4 of the radix-4 butterfly
template <bool INV, typename C>
__device__ __forceinline__ C frot(C a) {
    return INV ? fcx<C>(-a.y, a.x) : fcx<C>(a.y, -a.x);
}

// One radix-P butterfly: inputs src[q r] (q < P) times W_n^(q e), outputs dst[k1 Lr] (k1 < P).
// Odd P: the P-point DFT with the inputs taken in conjugate pairs (q, P - q), whose twiddles
// W_P^(q k) and W_P^((P - q) k) are conjugate: with S_q = a_q + a_{P-q}, D_q = a_q - a_{P-q} and
// W_P^(q k) = c + i s (W_P^j = W_n^(j n / P)),
//     b_k = X_k + i Y_k,  b_{P-k} = X_k - i Y_k,  X_k = a_0 + sum_q c S_q,  Y_k = sum_q s D_q,
// q, k = 1 .. (P - 1) / 2 (the inverse transform conjugates W: the two outputs swap).
template <int P, bool INV, typename C>
__device__ __forceinline__ void fft_butterfly(const C *src, C *dst, int r, int Lr, int e, const C *tw, int n) {
    C a[P];
#pragma unroll
    for (int q = 0; q < P; ++q) a[q] = q == 0 || e == 0 ? src[q * r] : fmulw<INV>(src[q * r], tw[q * e]);
    if constexpr (P == 2) {
        dst[0] = fadd(a[0], a[1]);
        dst[Lr] = fsub(a[0], a[1]);
    } else if constexpr (P == 4) {
        const C s02 = fadd(a[0], a[2]), d02 = fsub(a[0], a[2]);
        const C s13 = fadd(a[1], a[3]), d13 = frot<INV>(fsub(a[1], a[3]));
        dst[0] = fadd(s02, s13);
        dst[Lr] = fadd(d02, d13);
        dst[2 * Lr] = fsub(s02, s13);
        dst[3 * Lr] = fsub(d02, d13);
    } else {
        constexpr int H = (P - 1) / 2;
        const int step = n / P;
        C S[H + 1], D[H + 1];
        C b0 = a[0];
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            S[q] = fadd(a[q], a[P - q]);
            D[q] = fsub(a[q], a[P - q]);
            b0 = fadd(b0, S[q]);
        }
        dst[0] = b0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            C X = a[0], Y = fcx<C>(0, 0);
#pragma unroll
            for (int q = 1; q <= H; ++q) {
                const C w = tw[((q * k) % P) * step];
                X = fcx<C>(X.x + w.x * S[q].x, X.y + w.x * S[q].y);
                Y = fcx<C>(Y.x + w.y * D[q].x, Y.y + w.y * D[q].y);
            }
            const C iY = fcx<C>(-Y.y, Y.x);
            dst[k * Lr] = INV ? fsub(X, iY) : fadd(X, iY);
            dst[(P - k) * Lr] = INV ? fadd(X, iY) : fsub(X, iY);
        }
    }
}

// n-point transform by one warp: input in a, b the other buffer; returns the buffer that holds
// the result (natural order).  tw: W_n^j, j < n.
template <bool INV, typename C>
__device__ __noinline__ C *warp_fft(C *a, C *b, const FftPlan &P, const C *tw, int lane) {
    const int n = P.n;
    int L = 1;
    for (int s = 0; s < P.stages; ++s) {
        const int p = P.radix[s], r = n / (L * p), nb = n / p;
        for (int bi = lane; bi < nb; bi += 32) {
            const int k0 = bi / r, m = bi - k0 * r;
            const C *src = a + k0 * r * p + m;
            C *dst = b + k0 * r + m;
            const int e = k0 * r;  // W_{Lp}^(q k0) = W_n^(q k0 r)
            switch (p) {
                case 4: fft_butterfly<4, INV>(src, dst, r, L * r, e, tw, n); break;
                case 2: fft_butterfly<2, INV>(src, dst, r, L * r, e, tw, n); break;
                case 3: fft_butterfly<3, INV>(src, dst, r, L * r, e, tw, n); break;
                case 5: fft_butterfly<5, INV>(src, dst, r, L * r, e, tw, n); break;
                case 7: fft_butterfly<7, INV>(src, dst, r, L * r, e, tw, n); break;
                default: fft_butterfly<11, INV>(src, dst, r, L * r, e, tw, n); break;
            }
        }
        __syncwarp();
        C *t = a;
        a = b;
        b = t;
        L *= p;
    }
    return a;
}

// The same transform with the plan fixed at compile time (the paper's meshes 64, 88 and 128):
// every stage's radix, stride and butterfly count are constants, so the index arithmetic folds
// and the radix dispatch disappears.
struct CtPlan {
    int stages = 0;
    int radix[kFftMaxStages] = {};
};
__host__ __device__ constexpr CtPlan ct_plan(int n) {
    CtPlan p{};
    int m = n;
    const int rs[6] = {11, 7, 5, 3, 4, 2};
    for (int i = 0; i < 6; ++i)
        while (m % rs[i] == 0 && p.stages < kFftMaxStages) {
            p.radix[p.stages++] = rs[i];
            m /= rs[i];
        }
    return p;
}

template <int N, int S, int L, bool INV, typename C>
__device__ __forceinline__ C *ct_fft_stages(C *a, C *b, const C *tw, int lane) {
    constexpr CtPlan P = ct_plan(N);
    if constexpr (S == P.stages) {
        return a;
    } else {
        constexpr int p = P.radix[S], r = N / (L * p), nb = N / p;
#pragma unroll
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int bi = b0 + lane;
            if (nb % 32 == 0 || bi < nb) {
                const int k0 = bi / r, m = bi - k0 * r;
                fft_butterfly<p, INV>(a + k0 * r * p + m, b + k0 * r + m, r, L * r, k0 * r, tw, N);
            }
        }
        __syncwarp();
        return ct_fft_stages<N, S + 1, L * p, INV>(b, a, tw, lane);
    }
}

// n-point transform by one warp; N > 0: the compile-time plan of N (n == N), else P's.
template <int N, bool INV, typename C>
__device__ __forceinline__ C *warp_fft_any(C *a, C *b, const FftPlan &P, const C *tw, int lane) {
    if constexpr (N > 0) {
        static_assert(ct_plan(N).stages > 0, "no plan");
        return ct_fft_stages<N, 0, 1, INV>(a, b, tw, lane);
    } else {
        return warp_fft<INV>(a, b, P, tw, lane);
    }
}

// Shared memory of cta_disc_sums for an n x n lattice and `warps` warps: the half spectrum,
// then two buffers of n complex values per warp.
template <typename T>
__host__ __device__ constexpr size_t fft_smem_bytes(int n, int warps) {
    return ((size_t)n * (n / 2 + 1) + (size_t)warps * 2 * n) * sizeof(typename FftCx<T>::t);
}

// S = sum_{z in D} w_z u_{. + z} of one n x n sample by the whole CTA (n even).  ld(y, x) gives
// u; st(y, x, S) receives each sum once (rows in pairs, any order).  smem: fft_smem_bytes(n,
// warps of the CTA) bytes, 16-byte aligned; khat: K^(ky, kx) / n^2 at [ky][n/2 + 1] (global);
// tw: W_n^j, j < n (global).  Begins and ends with a CTA barrier, so smem may be shared with
// other phases of the caller.  N > 0: n == N, transformed with the compile-time plan.
template <int N, typename T, typename Ld, typename St>
__device__ __noinline__ void cta_disc_sums(const FftPlan &P, void *smem, const T *khat,
                                           const typename FftCx<T>::t *tw, Ld ld, St st) {
    using C = typename FftCx<T>::t;
    const int n = N > 0 ? N : P.n, NH = n / 2 + 1, nw = blockDim.x >> 5, w = threadIdx.x >> 5,
              lane = threadIdx.x & 31;
    C *spec = reinterpret_cast<C *>(smem);
    C *A = spec + (size_t)n * NH + (size_t)w * 2 * n, *B = A + n;
    const T half = T(0.5);
    __syncthreads();
    for (int pr = w; pr < n / 2; pr += nw) {  // forward row pass
        for (int x = lane; x < n; x += 32) A[x] = fcx<C>(ld(2 * pr, x), ld(2 * pr + 1, x));
        __syncwarp();
        const C *Z = warp_fft_any<N, false>(A, B, P, tw, lane);
        C *sa = spec + (size_t)(2 * pr) * NH, *sb = sa + NH;
        for (int k = lane; k <= n / 2; k += 32) {
            const C zk = Z[k], zm = Z[k == 0 ? 0 : n - k];
            sa[k] = fcx<C>(half * (zk.x + zm.x), half * (zk.y - zm.y));
            sb[k] = fcx<C>(half * (zk.y + zm.y), half * (zm.x - zk.x));
        }
        __syncwarp();
    }
    __syncthreads();
    for (int c = w; c < NH; c += nw) {  // column pass
        for (int ky = lane; ky < n; ky += 32) A[ky] = spec[(size_t)ky * NH + c];
        __syncwarp();
        C *Y = warp_fft_any<N, false>(A, B, P, tw, lane);
        for (int ky = lane; ky < n; ky += 32) {
            const T k = khat[(size_t)ky * NH + c];
            Y[ky] = fcx<C>(Y[ky].x * k, Y[ky].y * k);
        }
        __syncwarp();
        const C *X = warp_fft_any<N, true>(Y, Y == A ? B : A, P, tw, lane);
        for (int ky = lane; ky < n; ky += 32) spec[(size_t)ky * NH + c] = X[ky];
        __syncwarp();
    }
    __syncthreads();
    for (int pr = w; pr < n / 2; pr += nw) {  // inverse row pass
        const C *sa = spec + (size_t)(2 * pr) * NH, *sb = sa + NH;
        for (int k = lane; k < n; k += 32) {
            if (k <= n / 2) {
                const C a = sa[k], b = sb[k];
                A[k] = fcx<C>(a.x - b.y, a.y + b.x);
            } else {
                const C a = sa[n - k], b = sb[n - k];
                A[k] = fcx<C>(a.x + b.y, b.x - a.y);
            }
        }
        __syncwarp();
        const C *S = warp_fft_any<N, true>(A, B, P, tw, lane);
        for (int x = lane; x < n; x += 32) {
            const C s = S[x];
            st(2 * pr, x, s.x);
            st(2 * pr + 1, x, s.y);
        }
        __syncwarp();
    }
    __syncthreads();
}

}  // namespace mfmc
