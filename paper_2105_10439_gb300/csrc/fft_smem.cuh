// Radix-2 complex FFT in one thread block's shared memory, shared by the
// structured operators (DCT dictionary, FFT convolution): decimation in time,
// in place, bit-reversed input and natural-order output, twiddles
// e^{-2 pi i m / H} from a table.  Everything is in an anonymous namespace, so
// each translation unit gets its own copy.
#pragma once

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// e^{i pi num / den} (den a power of two, 0 <= num < 2 den: the angle is exact)
__device__ __forceinline__ float2 expi_pi(long long num, long long den) {
    float sn, cs;
    sincospif((float)num / (float)den, &sn, &cs);
    return make_float2(cs, sn);
}

__device__ __forceinline__ int brev(int m, int logH) { return (int)(__brev((unsigned)m) >> (32 - logH)); }

// In-place radix-2 FFT of the H = 2^logH points in s (bit-reversed input,
// natural-order output); forward uses e^{-2 pi i / H}, inverse its conjugate
// (no 1/H factor).  tw[m] = e^{-2 pi i m / H}, m < H/2.
__device__ void fft_smem(float2* s, int logH, const float2* __restrict__ tw, bool inverse) {
    const int H = 1 << logH;
    for (int ls = 1; ls <= logH; ++ls) {
        const int half = 1 << (ls - 1), step = H >> ls;
        for (int i = threadIdx.x; i < H / 2; i += blockDim.x) {
            const int pos = i & (half - 1);
            const int a = ((i >> (ls - 1)) << ls) + pos, b = a + half;
            float2 w = __ldg(tw + pos * step);
            if (inverse) w.y = -w.y;
            const float2 x = s[a], t = cmul(w, s[b]);
            s[a] = make_float2(x.x + t.x, x.y + t.y);
            s[b] = make_float2(x.x - t.x, x.y - t.y);
        }
        __syncthreads();
    }
}

// In-place bit-reversal permutation of the H = 2^logH points in s (pairs
// swapped once each: the permutation is an involution).
__device__ void bitrev_smem(float2* s, int logH) {
    const int H = 1 << logH;
    for (int m = threadIdx.x; m < H; m += blockDim.x) {
        const int r = brev(m, logH);
        if (m < r) {
            const float2 t = s[m];
            s[m] = s[r];
            s[r] = t;
        }
    }
    __syncthreads();
}

}  // namespace
