// Random-access roofline probe.  The walk, seed and search kernels are bound
// by dependent random reads of Occ blocks, which a streaming copy peak does not
// describe.  This probe measures what the memory system delivers for random
// 32/64/128-byte reads over a buffer much larger than L2:
//   independent -- every thread issues 4 reads at a time, addresses from a hash;
//   dependent   -- every thread follows a chain: the next address depends on
//                  the data just read (the access pattern of an LF walk), with
//                  a chosen number of chains per SM.
#include "common.cuh"

namespace rb3 {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finalizer
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

__global__ void k_probe_fill(uint32_t *__restrict__ buf, int64_t nwords, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords; i += (int64_t)gridDim.x * blockDim.x)
        buf[i] = (uint32_t)mix64(seed ^ (uint64_t)i);
}

template <int NSEC, bool H64> __device__ __forceinline__ uint32_t read_unit(const uint8_t *p) {
    uint32_t acc = 0;
    Sec s[NSEC];
#pragma unroll
    for (int j = 0; j < NSEC; ++j) s[j] = H64 ? ld_sec64(p + 32 * j) : ld_sec(p + 32 * j);
#pragma unroll
    for (int j = 0; j < NSEC; ++j) acc ^= s[j].w[0] + s[j].w[7];
    return acc;
}

template <int NSEC, bool H64>
__global__ void k_probe_indep(const uint8_t *__restrict__ buf, uint64_t nunits, int iters, uint64_t seed,
                              uint32_t *__restrict__ sink) {
    uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < iters; i += 4) {
        uint64_t u[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) u[j] = mix64(seed ^ (t * (uint64_t)iters + i + j)) % nunits;
        uint32_t v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = read_unit<NSEC, H64>(buf + u[j] * (32 * NSEC));
        acc += v[0] ^ v[1] ^ v[2] ^ v[3];
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

template <int NSEC, bool H64>
__global__ void k_probe_chain(const uint8_t *__restrict__ buf, uint64_t nunits, int steps, uint64_t seed,
                              uint32_t *__restrict__ sink) {
    uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    uint64_t u = mix64(seed ^ t) % nunits;
    uint32_t acc = 0;
    for (int s = 0; s < steps; ++s) {
        uint32_t v = read_unit<NSEC, H64>(buf + u * (32 * NSEC));
        acc += v;
        u = mix64(u ^ v ^ (uint64_t)s) % nunits;
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

// Modes 4 / 5: modes 0 / 1 with a 64-byte L2 fetch-size hint on every read.
//
// Cooperative forms: the NSEC lanes of a group read the NSEC sectors of one
// unit in the same instruction (one request per unit instead of one per
// sector).  Dependent: the group's next address comes from the data of all
// its lanes (shuffled together).
template <int NSEC>
__global__ void k_probe_coop(const uint8_t *__restrict__ buf, uint64_t nunits, int iters, int dependent, uint64_t seed,
                             uint32_t *__restrict__ sink) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t grp = t / NSEC;
    const int sub = (int)(t % NSEC);
    uint32_t acc = 0;
    uint64_t u = mix64(seed ^ grp) % nunits;
    for (int i = 0; i < iters; ++i) {
        if (!dependent) u = mix64(seed ^ (grp * (uint64_t)iters + i)) % nunits;
        Sec s = ld_sec(buf + u * (32 * NSEC) + 32 * sub);
        uint32_t v = s.w[0] + s.w[7];
#pragma unroll
        for (int d = 1; d < NSEC; d <<= 1) v ^= __shfl_xor_sync(0xffffffffu, v, d, NSEC);
        acc += v;
        if (dependent) u = mix64(u ^ v ^ (uint64_t)i) % nunits;
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

int probe_random_gather(int bytes, int dependent, int threads_per_sm, int64_t buffer_bytes, double *gbs,
                        double *maccess, cudaStream_t st) {
    RB3_CHECK_ARG(bytes == 32 || bytes == 64 || bytes == 128, "bytes must be 32, 64 or 128");
    RB3_CHECK_ARG(dependent >= 0 && dependent <= 5, "mode must be 0..5");
    RB3_CHECK_ARG(threads_per_sm >= 32 && threads_per_sm <= 2048 && threads_per_sm % 32 == 0,
                  "threads_per_sm must be a multiple of 32 in [32, 2048]");
    RB3_CHECK_ARG(buffer_bytes >= (int64_t)(1 << 26), "buffer must be at least 64 MiB");
    DevBuf buf, sink;
    RB3_TRY(buf.alloc((size_t)buffer_bytes, st));
    RB3_TRY(sink.alloc(sizeof(uint32_t), st));
    int64_t nwords = buffer_bytes / 4;
    RB3_LAUNCH(k_probe_fill, (unsigned)(num_sms() * 8), 256, 0, st, buf.as<uint32_t>(), nwords, 0x51ull);
    const uint64_t nunits = (uint64_t)(buffer_bytes / bytes);
    const int block = threads_per_sm < 256 ? threads_per_sm : 256;
    const unsigned grid = (unsigned)((int64_t)num_sms() * threads_per_sm / block);
    const int64_t threads = (int64_t)grid * block;
    const int iters = (dependent == 1 || dependent == 3 || dependent == 5) ? 256 : 512;
    cudaEvent_t a, b;
    RB3_CUDA_TRY(cudaEventCreate(&a));
    RB3_CUDA_TRY(cudaEventCreate(&b));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        RB3_CUDA_TRY(cudaEventRecord(a, st));
        const uint8_t *p = buf.as<uint8_t>();
        uint32_t *s = sink.as<uint32_t>();
        uint64_t seed = 1000 + rep;
        if (dependent == 2 || dependent == 3) {  // cooperative: 2 = independent, 3 = dependent
            const int dep = dependent == 3;
            if (bytes == 32) RB3_LAUNCH(k_probe_coop<1>, grid, block, 0, st, p, nunits, iters, dep, seed, s);
            else if (bytes == 64) RB3_LAUNCH(k_probe_coop<2>, grid, block, 0, st, p, nunits, iters, dep, seed, s);
            else RB3_LAUNCH(k_probe_coop<4>, grid, block, 0, st, p, nunits, iters, dep, seed, s);
        } else if (dependent == 1 || dependent == 5) {
            if (dependent == 5) {
                if (bytes == 32) RB3_LAUNCH((k_probe_chain<1, true>), grid, block, 0, st, p, nunits, iters, seed, s);
                else if (bytes == 64) RB3_LAUNCH((k_probe_chain<2, true>), grid, block, 0, st, p, nunits, iters, seed, s);
                else RB3_LAUNCH((k_probe_chain<4, true>), grid, block, 0, st, p, nunits, iters, seed, s);
            } else {
                if (bytes == 32) RB3_LAUNCH((k_probe_chain<1, false>), grid, block, 0, st, p, nunits, iters, seed, s);
                else if (bytes == 64) RB3_LAUNCH((k_probe_chain<2, false>), grid, block, 0, st, p, nunits, iters, seed, s);
                else RB3_LAUNCH((k_probe_chain<4, false>), grid, block, 0, st, p, nunits, iters, seed, s);
            }
        } else {
            if (dependent == 4) {
                if (bytes == 32) RB3_LAUNCH((k_probe_indep<1, true>), grid, block, 0, st, p, nunits, iters, seed, s);
                else if (bytes == 64) RB3_LAUNCH((k_probe_indep<2, true>), grid, block, 0, st, p, nunits, iters, seed, s);
                else RB3_LAUNCH((k_probe_indep<4, true>), grid, block, 0, st, p, nunits, iters, seed, s);
            } else {
                if (bytes == 32) RB3_LAUNCH((k_probe_indep<1, false>), grid, block, 0, st, p, nunits, iters, seed, s);
                else if (bytes == 64) RB3_LAUNCH((k_probe_indep<2, false>), grid, block, 0, st, p, nunits, iters, seed, s);
                else RB3_LAUNCH((k_probe_indep<4, false>), grid, block, 0, st, p, nunits, iters, seed, s);
            }
        }
        RB3_CUDA_TRY(cudaEventRecord(b, st));
        RB3_CUDA_TRY(cudaEventSynchronize(b));
        float ms = 0.f;
        RB3_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    double accesses = (double)threads * iters;
    if (dependent == 2 || dependent == 3) accesses /= (bytes / 32);  // one access per lane group
    if (gbs) *gbs = accesses * bytes / (best * 1e-3) / 1e9;
    if (maccess) *maccess = accesses / (best * 1e-3) / 1e6;
    return RB3_OK;
}

}  // namespace rb3

RB3_EXPORT int rb3_probe_random_gather(int32_t bytes_per_access, int32_t dependent, int32_t threads_per_sm,
                                       int64_t buffer_bytes, double *gbs, double *maccess_per_s, void *stream) {
    return rb3::probe_random_gather(bytes_per_access, dependent, threads_per_sm, buffer_bytes, gbs, maccess_per_s,
                                    (cudaStream_t)stream);
}
