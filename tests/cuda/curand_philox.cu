// Test harness: Philox4x32-10 blocks from cuRAND's device API, used to pin the
// oracle's and the library's generator against an independent implementation.
// Reads lines "key_lo key_hi c0 c1 c2 c3" (decimal) on stdin and prints the four
// output words of the block at that counter.  cuRAND's state is positioned with
// curand_init(seed, subsequence, offset): the block counter is
// (offset / 4 low, high, subsequence low, high); offset counts 32-bit outputs, so
// the counter's high word c1 must stay below 2^30.
#include <cstdio>
#include <cstdint>
#include <vector>
#include <curand_kernel.h>

__global__ void blocks(const unsigned long long* in, unsigned int* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long seed = in[3 * i];
    const unsigned long long offset_blocks = in[3 * i + 1];
    const unsigned long long subseq = in[3 * i + 2];
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq, offset_blocks * 4ull, &st);
    const uint4 v = curand4(&st);
    out[4 * i + 0] = v.x;
    out[4 * i + 1] = v.y;
    out[4 * i + 2] = v.z;
    out[4 * i + 3] = v.w;
}

int main() {
    std::vector<unsigned long long> in;
    unsigned long long klo, khi, c0, c1, c2, c3;
    while (std::scanf("%llu %llu %llu %llu %llu %llu", &klo, &khi, &c0, &c1, &c2, &c3) == 6) {
        in.push_back(klo | (khi << 32));
        in.push_back(c0 | (c1 << 32));
        in.push_back(c2 | (c3 << 32));
    }
    const int n = (int)(in.size() / 3);
    if (n == 0) return 0;
    unsigned long long* d_in = nullptr;
    unsigned int* d_out = nullptr;
    if (cudaMalloc(&d_in, in.size() * sizeof(unsigned long long)) != cudaSuccess) return 2;
    if (cudaMalloc(&d_out, (size_t)n * 4 * sizeof(unsigned int)) != cudaSuccess) return 2;
    cudaMemcpy(d_in, in.data(), in.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    blocks<<<(n + 127) / 128, 128>>>(d_in, d_out, n);
    std::vector<unsigned int> out((size_t)n * 4);
    if (cudaMemcpy(out.data(), d_out, out.size() * sizeof(unsigned int), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    for (int i = 0; i < n; ++i) std::printf("%u %u %u %u\n", out[4 * i], out[4 * i + 1], out[4 * i + 2], out[4 * i + 3]);
    cudaFree(d_in);
    cudaFree(d_out);
    return 0;
}
