// Prints cuRAND's Philox4_32_10 output for the counters and keys read from
// stdin ("c0 c1 c2 c3 k0 k1" per line), one line of four words per input.
// The first curand4() after curand_init(seed, subsequence, offset) returns
// Philox(counter = (offset/4 as 64 bits, subsequence as 64 bits), key = seed).
#include <cstdio>
#include <vector>
#include <curand_kernel.h>

__global__ void run(const unsigned *in, unsigned *out, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned *q = in + 6 * i;
    unsigned long long seed = ((unsigned long long)q[5] << 32) | q[4];
    unsigned long long sub = ((unsigned long long)q[3] << 32) | q[2];
    unsigned long long off = (((unsigned long long)q[1] << 32) | q[0]) * 4ull;
    curandStatePhilox4_32_10_t s;
    curand_init(seed, sub, off, &s);
    uint4 r = curand4(&s);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

int main()
{
    std::vector<unsigned> in;
    unsigned v[6];
    while (scanf("%u %u %u %u %u %u", v, v + 1, v + 2, v + 3, v + 4, v + 5) == 6) in.insert(in.end(), v, v + 6);
    int n = (int)(in.size() / 6);
    if (n == 0) return 1;
    unsigned *di, *dout;
    if (cudaMalloc(&di, in.size() * 4) != cudaSuccess) return 2;
    if (cudaMalloc(&dout, (size_t)n * 16) != cudaSuccess) return 2;
    cudaMemcpy(di, in.data(), in.size() * 4, cudaMemcpyHostToDevice);
    run<<<(n + 127) / 128, 128>>>(di, dout, n);
    std::vector<unsigned> out((size_t)n * 4);
    if (cudaMemcpy(out.data(), dout, out.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
    for (int i = 0; i < n; ++i) printf("%u %u %u %u\n", out[4 * i], out[4 * i + 1], out[4 * i + 2], out[4 * i + 3]);
    cudaFree(di);
    cudaFree(dout);
    return 0;
}
