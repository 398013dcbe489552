// selftest_curand.cu -- test-support library (libfpt_selftest.so), not part of the engine.
//
// Produces the output words of cuRAND's device Philox4_32_10 generator so that the engine's own
// Philox4x32-10 can be compared with an independent implementation on the GPU.  cuRAND seeds a
// stream with key = seed and counter = (0, 0, subsequence lo, subsequence hi) and hands out the
// four words of each counter value in order; the engine's block b of trajectory t is therefore
// cuRAND's (seed, subsequence = t, offset = 4 b).
#include <curand_kernel.h>

namespace {

__global__ void curand_philox_kernel(unsigned long long seed, unsigned long long subseq0,
                                     unsigned long long offset, unsigned nseq, unsigned nwords,
                                     unsigned *out) {
    const unsigned j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nseq) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq0 + j, offset, &st);
    for (unsigned i = 0; i < nwords; ++i) out[static_cast<size_t>(j) * nwords + i] = curand(&st);
}

}  // namespace

// nseq consecutive subsequences, nwords words each starting at `offset`, into d_out
// (device, nseq * nwords uint32).  Returns the cudaError_t of the launch and synchronisation.
extern "C" int fpt_selftest_curand_philox(unsigned long long seed, unsigned long long subseq0,
                                          unsigned long long offset, unsigned nseq,
                                          unsigned nwords, unsigned *d_out) {
    if (nseq == 0 || nwords == 0) return 0;
    curand_philox_kernel<<<(nseq + 127) / 128, 128>>>(seed, subseq0, offset, nseq, nwords, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return static_cast<int>(e);
    return static_cast<int>(cudaDeviceSynchronize());
}
