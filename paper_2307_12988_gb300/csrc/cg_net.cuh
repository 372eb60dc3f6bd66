// cg_net.cuh -- compile-time comparator networks for selection in registers.
//
// OddEvenNet<N>: Batcher's odd-even merge sort on N = 2^m wires (Knuth,
// TAOCP vol. 3, 5.3.4), as a list of comparators (lo, hi): after each one,
// wire lo holds the smaller and wire hi the larger of the two values.
//
// RankNet<N, NREAL, RANK, RANK2>: that network reduced to what the outputs
// RANK and RANK2 (the RANK-th and RANK2-th smallest, from 0, of NREAL
// values) need, when wires NREAL..N-1 hold +infinity:
//   * a forward pass follows the infinite pads: a comparator with an infinite
//     hi input changes nothing (dropped); one with an infinite lo input only
//     moves the hi value down (a register move, kept as a move);
//   * a backward pass from the output keeps only comparators one of whose
//     outputs is needed, and of those computes only the needed output (min
//     alone, max alone, or both).
// Every kept step moves or compares values without arithmetic, so the result
// is one of the inputs, exactly.
#pragma once

namespace cg {

template <int N>
struct OddEvenNet {
    static constexpr int count_()
    {
        int c = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k && i + j + k < N; ++i)
                        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) ++c;
        return c;
    }
    static constexpr int kCount = count_();
    int lo[kCount], hi[kCount];
    constexpr OddEvenNet() : lo(), hi()
    {
        int c = 0;
        for (int p = 1; p < N; p <<= 1)
            for (int k = p; k >= 1; k >>= 1)
                for (int j = k % p; j + k < N; j += 2 * k)
                    for (int i = 0; i < k && i + j + k < N; ++i)
                        if ((i + j) / (2 * p) == (i + j + k) / (2 * p)) {
                            lo[c] = i + j;
                            hi[c] = i + j + k;
                            ++c;
                        }
    }
};

// step kinds of RankNet
enum : int { kNetSkip = 0, kNetMin = 1, kNetMax = 2, kNetBoth = 3, kNetMove = 4 };

template <int N, int NREAL, int RANK, int RANK2 = RANK>
struct RankNet {
    static constexpr int kCount = OddEvenNet<N>::kCount;
    int lo[kCount], hi[kCount], kind[kCount];
    constexpr RankNet() : lo(), hi(), kind()
    {
        constexpr OddEvenNet<N> net{};
        bool inf[N] = {};
        for (int w = 0; w < N; ++w) inf[w] = w >= NREAL;
        // forward: the infinite pads
        for (int c = 0; c < kCount; ++c) {
            const int l = net.lo[c], h = net.hi[c];
            lo[c] = l;
            hi[c] = h;
            if (inf[h]) {
                kind[c] = kNetSkip;   // min is lo's value, max stays infinite
            } else if (inf[l]) {
                kind[c] = kNetMove;   // lo takes hi's value, hi becomes infinite
                inf[l] = false;
                inf[h] = true;
            } else {
                kind[c] = kNetBoth;
            }
        }
        // backward: what the output needs
        bool need[N] = {};
        need[RANK] = true;
        need[RANK2] = true;
        for (int c = kCount - 1; c >= 0; --c) {
            const int l = lo[c], h = hi[c];
            if (kind[c] == kNetMove) {
                if (need[l]) {
                    need[h] = true;
                    need[l] = false;
                } else {
                    kind[c] = kNetSkip;
                }
            } else if (kind[c] == kNetBoth) {
                const int k = (need[l] ? kNetMin : 0) | (need[h] ? kNetMax : 0);
                kind[c] = k;
                if (k != kNetSkip) need[l] = need[h] = true;
            }
        }
    }
};

// Leaves the RANK-th and RANK2-th smallest of v[0..NREAL) in v[RANK] and
// v[RANK2] (v[NREAL..N) are not read; the other entries are clobbered).
template <int N, int NREAL, int RANK, int RANK2 = RANK>
__device__ __forceinline__ void rank_network(float (&v)[N])
{
    constexpr RankNet<N, NREAL, RANK, RANK2> net{};
#pragma unroll
    for (int c = 0; c < RankNet<N, NREAL, RANK, RANK2>::kCount; ++c) {
        const int l = net.lo[c], h = net.hi[c];
        if (net.kind[c] == kNetBoth) {
            const float a = v[l], b = v[h];
            v[l] = fminf(a, b);
            v[h] = fmaxf(a, b);
        } else if (net.kind[c] == kNetMin) {
            v[l] = fminf(v[l], v[h]);
        } else if (net.kind[c] == kNetMax) {
            v[h] = fmaxf(v[l], v[h]);
        } else if (net.kind[c] == kNetMove) {
            v[l] = v[h];
        }
    }
}

// RANK-th smallest of v[0..NREAL) (v[NREAL..N) are not read); v is clobbered.
template <int N, int NREAL, int RANK>
__device__ __forceinline__ float rank_select(float (&v)[N])
{
    rank_network<N, NREAL, RANK>(v);
    return v[RANK];
}

}  // namespace cg
