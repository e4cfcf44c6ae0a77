// Grid-wide synchronisation and fixed-order reductions for persistent
// cooperative kernels (all CTAs co-resident).
//
// grid_sync: counter + generation barrier with a bounded spin; a CTA that
// gives up sets the error flag, and every waiting CTA returns as soon as it
// sees the flag, so no launch can wait forever.
// block_sum_t / write_partial / sum_partials: per-CTA partial sums written to
// global memory before the barrier and summed after it by every CTA in the
// same order, so all CTAs take identical decisions from identical values.
#pragma once
#include <cuda_runtime.h>

namespace wmg {

constexpr long long kBarrierSpinLimit = 40000000LL;   // a few seconds of polls

__device__ __forceinline__ bool grid_sync(unsigned int* count, unsigned int* gen, unsigned int G, int* err,
                                          long long limit = kBarrierSpinLimit) {
    __shared__ int s_fail;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_fail = 0;
        volatile unsigned int* vgen = gen;
        volatile int* verr = err;
        unsigned int my = *vgen;
        __threadfence();
        if (atomicAdd(count, 1u) == G - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == my) {
                if (*verr) { s_fail = 1; break; }
                if (++spins > limit) { atomicExch(err, 1); s_fail = 1; break; }
                if (spins > 256) __nanosleep(32);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_fail == 0;
}

template <typename T> __device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// CTA sum in precision T (fixed order), valid in every thread
template <typename T> __device__ __forceinline__ T block_sum_t(T v, T* sh) {
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_t(v);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T x = lane < nw ? sh[lane] : T(0);
        x = warp_sum_t(x);
        if (lane == 0) sh[32] = x;
    }
    __syncthreads();
    T r = sh[32];
    __syncthreads();
    return r;
}
// sum of partials[c * 4 + slot] over c < G in a fixed order, broadcast to the CTA
template <typename T> __device__ __forceinline__ T sum_partials(const double* partials, int slot, int G, T* sh) {
    T a = 0;
    for (int c = threadIdx.x; c < G; c += blockDim.x) a += (T)__ldcg(partials + (size_t)c * 4 + slot);
    return block_sum_t<T>(a, sh);
}
template <typename T> __device__ __forceinline__ void write_partial(T v, double* partials, int slot, T* sh) {
    T a = block_sum_t<T>(v, sh);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.x * 4 + slot] = (double)a;
}


// ---------------------------------------------------------------- epoch exchange
// All-to-all exchange of per-CTA partial sums that is also the grid barrier:
// CTA c publishes (value, epoch) as one 8-byte word in its slot (a release at
// GPU scope by thread 0, after a CTA barrier, so every global write the CTA made
// before is ordered before it), and every CTA waits, one thread per slot, until
// all G slots carry the epoch (acquire), then sums the values in CTA order.
// Slots are double-buffered by epoch parity: a CTA can be at most one exchange
// ahead of the slowest one, so it never overwrites a word another CTA still
// waits for.  Epochs increase across launches (the host reserves a range per
// launch and clears the slots when the 32-bit counter would wrap).
constexpr long long kExchangeSpinLimit = 40000000LL;   // a few seconds of polls

__device__ __forceinline__ void xch_publish(unsigned long long* slot, float v, unsigned int e) {
    const unsigned long long w = ((unsigned long long)e << 32) | __float_as_uint(v);
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(slot), "l"(w) : "memory");
}
// relaxed publish: for callers whose shared data carries its own epoch tags
// (nothing else has to be visible when the value is)
__device__ __forceinline__ void xch_publish_relaxed(unsigned long long* slot, float v, unsigned int e) {
    const unsigned long long w = ((unsigned long long)e << 32) | __float_as_uint(v);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(slot), "l"(w) : "memory");
}
__device__ __forceinline__ unsigned long long xch_load(const unsigned long long* slot) {
    unsigned long long w;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(slot) : "memory");
    return w;
}
// bounded wait until *slot carries epoch e; false on timeout or a raised error flag
__device__ __forceinline__ bool xch_wait(const unsigned long long* slot, unsigned int e, int* err, float& v,
                                         long long limit = kExchangeSpinLimit) {
    long long spins = 0;
    for (;;) {
        const unsigned long long w = xch_load(slot);
        if ((unsigned int)(w >> 32) == e) {
            v = __uint_as_float((unsigned int)w);
            return true;
        }
        if (*(volatile int*)err) return false;
        if (++spins > limit) {
            atomicExch(err, 1);
            return false;
        }
        if (spins > 32) __nanosleep(20);
    }
}
// Each slot sits alone in a 128-byte line (kXchPad words): every slot is polled
// by one thread of every CTA, and slots packed into a few lines made those lines
// a hot spot (measured: 4.2 us from the last publish to the first CTA through,
// 2.3 us with one slot per line).
constexpr int kXchPad = 16;
constexpr int kXchMaxNV = 3;
// v[j] (this thread's share) -> the grid-wide sums, identical in every CTA.
// slots: [parity 2][value kXchMaxNV][G][kXchPad]; the parity is that of e, so
// consecutive calls must use consecutive epochs.
// sc: shared scratch of at least NV * (32 + G + 1) floats, free during the call.
// Three CTA barriers for any NV: warp partial sums -> thread 0 publishes;
// polled values -> one warp per value sums them in CTA order.
// FENCE false: no fence before the publish (the caller's cross-CTA data is
// epoch-tagged, so only the partial sums themselves must arrive).
// Gx: the number of CTAs that publish (0: gridDim.x); limit: polls per slot.
// The exchange in two halves, so that a caller can do independent work between
// publishing its share and collecting the sums: xch_post (warp partial sums,
// one CTA barrier, thread 0 publishes) and xch_collect (poll, sum; two CTA
// barriers).  The scratch sc must stay untouched from xch_post to xch_collect.
template <int NV, bool FENCE = true>
__device__ void xch_post(const float (&v)[NV], unsigned long long* slots, unsigned int e, float* sc, int Gx = 0) {
    static_assert(NV >= 1 && NV <= kXchMaxNV, "one to three values per exchange");
    const int G = Gx > 0 ? Gx : (int)gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    unsigned long long* base = slots + (size_t)(e & 1) * kXchMaxNV * G * kXchPad;
    float* wsum = sc;                  // [NV][32] warp partials
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const float w = warp_sum_t<float>(v[j]);
        if (lane == 0) wsum[j * 32 + warp] = w;
    }
    __syncthreads();
    if (t == 0) {
        float cta[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float a = 0.f;
            for (int i = 0; i < nw; ++i) a += wsum[j * 32 + i];
            cta[j] = a;
        }
        if (FENCE) {
            __threadfence();
#pragma unroll
            for (int j = 0; j < NV; ++j) xch_publish(base + ((size_t)j * G + blockIdx.x) * kXchPad, cta[j], e);
        } else {
#pragma unroll
            for (int j = 0; j < NV; ++j) xch_publish_relaxed(base + ((size_t)j * G + blockIdx.x) * kXchPad, cta[j], e);
        }
    }
}
template <int NV>
__device__ bool xch_collect(float (&v)[NV], const unsigned long long* slots, unsigned int e, int* err, float* sc,
                            int Gx = 0, long long limit = kExchangeSpinLimit) {
    const int G = Gx > 0 ? Gx : (int)gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned long long* base = slots + (size_t)(e & 1) * kXchMaxNV * G * kXchPad;
    float* gv = sc + NV * 32;          // [NV * G] polled CTA sums
    float* res = gv + NV * G;          // [NV] grid sums
    bool ok = true;
    for (int i = t; i < NV * G && ok; i += blockDim.x) {
        float got = 0.f;
        ok = xch_wait(base + (size_t)i * kXchPad, e, err, got, limit);
        gv[i] = got;
    }
    if (__syncthreads_or(!ok)) return false;
    if (warp < NV) {
        float a = 0.f;
        for (int c = lane; c < G; c += 32) a += gv[warp * G + c];
        a = warp_sum_t<float>(a);
        if (lane == 0) res[warp] = a;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = res[j];
    return true;
}
// Packed form for callers whose cross-CTA data carries its own epoch tags (so
// the exchange orders nothing but its own values): a CTA's NV partial sums sit
// in one 128-byte line, words 0..NV-1 each (epoch << 32 | value), stored and
// polled with relaxed GPU-scope accesses, one polling thread per CTA line.
// slots: [parity 2][G][kXchPad] (inside the unpacked layout's footprint);
// epochs consecutive as for xch_post.  Every word is single-copy atomic, and
// the reader re-polls until all NV words carry the epoch.
__device__ __forceinline__ void xch_store_words(unsigned long long* line, const unsigned long long* w, int n) {
    if (n >= 2)
        asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(line), "l"(w[0]), "l"(w[1]) : "memory");
    else
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(line), "l"(w[0]) : "memory");
    if (n == 3) asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(line + 2), "l"(w[2]) : "memory");
}
template <int NV>
__device__ void xch_post_packed(const float (&v)[NV], unsigned long long* slots, unsigned int e, float* sc) {
    static_assert(NV >= 1 && NV <= kXchMaxNV, "one to three values per exchange");
    const int G = (int)gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    unsigned long long* line = slots + ((size_t)(e & 1) * G + blockIdx.x) * kXchPad;
    float* wsum = sc;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const float w = warp_sum_t<float>(v[j]);
        if (lane == 0) wsum[j * 32 + warp] = w;
    }
    __syncthreads();
    if (t == 0) {
        unsigned long long w[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            float a = 0.f;
            for (int i = 0; i < nw; ++i) a += wsum[j * 32 + i];
            w[j] = ((unsigned long long)e << 32) | __float_as_uint(a);
        }
        xch_store_words(line, w, NV);
    }
}
template <int NV>
__device__ bool xch_collect_packed(float (&v)[NV], const unsigned long long* slots, unsigned int e, int* err, float* sc,
                                   long long limit = kExchangeSpinLimit) {
    const int G = (int)gridDim.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned long long* base = slots + (size_t)(e & 1) * G * kXchPad;
    float* gv = sc + NV * 32;          // [NV][G] polled CTA sums
    float* res = gv + NV * G;          // [NV] grid sums
    bool ok = true;
    for (int c = t; c < G && ok; c += blockDim.x) {
        const unsigned long long* line = base + (size_t)c * kXchPad;
        long long spins = 0;
        for (;;) {
            unsigned long long w[3] = {0ull, 0ull, 0ull};
            if (NV >= 2)
                asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(line) : "memory");
            else
                asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w[0]) : "l"(line) : "memory");
            if (NV == 3) asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(w[2]) : "l"(line + 2) : "memory");
            bool all = true;
#pragma unroll
            for (int j = 0; j < NV; ++j) all = all && (unsigned int)(w[j] >> 32) == e;
            if (all) {
#pragma unroll
                for (int j = 0; j < NV; ++j) gv[j * G + c] = __uint_as_float((unsigned int)w[j]);
                break;
            }
            if (*(volatile int*)err) { ok = false; break; }
            if (++spins > limit) {
                atomicExch(err, 1);
                ok = false;
                break;
            }
            if (spins > 32) __nanosleep(20);
        }
    }
    if (__syncthreads_or(!ok)) return false;
    if (warp < NV) {
        float a = 0.f;
        for (int c = lane; c < G; c += 32) a += gv[warp * G + c];
        a = warp_sum_t<float>(a);
        if (lane == 0) res[warp] = a;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = res[j];
    return true;
}

// v[j] (this thread's share) -> the grid-wide sums, identical in every CTA.
// slots: [parity 2][value kXchMaxNV][G][kXchPad]; the parity is that of e, so
// consecutive calls must use consecutive epochs.
// sc: shared scratch of at least NV * (32 + G + 1) floats, free during the call.
// Three CTA barriers for any NV: warp partial sums -> thread 0 publishes;
// polled values -> one warp per value sums them in CTA order.
// FENCE false: no fence before the publish (the caller's cross-CTA data is
// epoch-tagged, so only the partial sums themselves must arrive).
// Gx: the number of CTAs that publish (0: gridDim.x); limit: polls per slot.
template <int NV, bool FENCE = true>
__device__ bool xch_allreduce(float (&v)[NV], unsigned long long* slots, unsigned int e, int* err, float* sc, int Gx = 0,
                              long long limit = kExchangeSpinLimit) {
    xch_post<NV, FENCE>(v, slots, e, sc, Gx);
    return xch_collect<NV>(v, slots, e, err, sc, Gx, limit);
}

// ---------------------------------------------------------------- epoch-tagged vectors
// A complex entry as two 64-bit words (epoch << 32 | float bits) for re and im.
// Each word is written and read whole (single-copy atomic), so a reader that
// sees the expected epoch in both words has the value of that epoch, with no
// fence or flag between writer and reader.
__device__ __forceinline__ void tag_store(unsigned long long* w, float re, float im, unsigned int e) {
    const unsigned long long a = ((unsigned long long)e << 32) | __float_as_uint(re);
    const unsigned long long b = ((unsigned long long)e << 32) | __float_as_uint(im);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(w), "l"(a), "l"(b) : "memory");
}
// one load; true when both words carry epoch e
__device__ __forceinline__ bool tag_load(const unsigned long long* w, unsigned int e, float2& v) {
    unsigned long long a, b;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(w) : "memory");
    v = make_float2(__uint_as_float((unsigned int)a), __uint_as_float((unsigned int)b));
    return (unsigned int)(a >> 32) == e && (unsigned int)(b >> 32) == e;
}
// bounded wait for epoch e at w; false on timeout or a raised error flag
__device__ __forceinline__ bool tag_wait(const unsigned long long* w, unsigned int e, int* err, float2& v,
                                         long long limit = kExchangeSpinLimit) {
    long long spins = 0;
    while (!tag_load(w, e, v)) {
        if (*(volatile int*)err) return false;
        if (++spins > limit) {
            atomicExch(err, 1);
            return false;
        }
        if (spins > 32) __nanosleep(20);
    }
    return true;
}

}  // namespace wmg
