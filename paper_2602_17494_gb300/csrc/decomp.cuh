// One axis of the overlapping decomposition of Section 6.1.
//
// Reading of the paper (which fixes only the properties of theta): the cores
// split an axis of N image pixels as evenly as integers allow, core k =
// [floor(kN/M), floor((k+1)N/M)); neighbouring subdomains share a strip of s
// pixels [b - ceil(s/2), b + floor(s/2)) around their core boundary b, on
// which theta falls (lower subdomain) or rises (upper subdomain) linearly,
// evaluated at pixel centres; theta = 1 elsewhere in a subdomain.  The grid
// may be longer than N (the extended grid has N + 1 points); the extra points
// belong to the last subdomain, so both steps share the same cores.
#pragma once

struct Axis {
    int N, M, s;   // image pixels on the axis, subdomains, overlap
    int L;         // grid points on the axis (N, or N + 1 for the extended grid)
    __host__ __device__ __forceinline__ int core(int k) const {
        // k <= M <= N < 2^16 keeps k N in 32 bits; wider axes take the 64-bit path
        if (N < 65536) return (int)(((unsigned)k * (unsigned)N) / (unsigned)M);
        return (int)(((long long)k * N) / M);
    }
    __host__ __device__ __forceinline__ int start(int k) const { return k == 0 ? 0 : core(k) - (s + 1) / 2; }
    __host__ __device__ __forceinline__ int end(int k) const { return k == M - 1 ? L : core(k + 1) + s / 2; }
    // theta of part k at grid point x (x inside [start(k), end(k)))
    __host__ __device__ __forceinline__ float theta(int k, int x) const {
        const int lo = (s + 1) / 2;
        if (s > 0 && k > 0) {
            const int a = core(k) - lo;
            if (x < a + s) return ((float)(x - a) + 0.5f) / (float)s;
        }
        if (s > 0 && k < M - 1) {
            const int a = core(k + 1) - lo;
            if (x >= a) return ((float)(a + s - x) - 0.5f) / (float)s;
        }
        return 1.0f;
    }
    __host__ __device__ __forceinline__ float theta_or0(int k, int x) const {
        return (x >= start(k) && x < end(k)) ? theta(k, x) : 0.0f;
    }
    __host__ __device__ __forceinline__ int core_of(int x) const {
        int k = (int)(((long long)x * M) / N);
        if (k > M - 1) k = M - 1;
        while (k + 1 < M && core(k + 1) <= x) ++k;
        while (k > 0 && core(k) > x) --k;
        return k;
    }
};
