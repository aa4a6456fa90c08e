// Checks the bounded mbarrier wait of async_copy.cuh: a barrier that nothing
// completes makes mbar_wait give up after its poll limit and return false
// (the kernels turn that into an error flag instead of spinning), a barrier
// completed by an arrival makes it return true, and the context stays usable
// afterwards.  Prints the outcomes and the time of the expired wait.
#include <cstdint>
#include <cstdio>

#include "async_copy.cuh"

using sdc::mbar_init;
using sdc::mbar_init_fence;
using sdc::mbar_wait;

__global__ void wait_on_barrier(int arrive, int *out) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sdc::smem_u32(&bar)) : "memory");
    const bool done = mbar_wait(&bar, 0);
    if (threadIdx.x == 0) out[0] = done ? 1 : 0;
}

__global__ void add_one(int *x) { x[threadIdx.x] += 1; }

int main() {
    int *d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(int)) != cudaSuccess) return 2;
    cudaMemset(d, 0, 4 * sizeof(int));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a);
    wait_on_barrier<<<1, 32>>>(0, d);          // nothing completes the phase
    cudaEventRecord(b);
    wait_on_barrier<<<1, 32>>>(1, d + 1);      // one arrival completes it
    add_one<<<1, 2>>>(d + 2);
    int h[4] = {-1, -1, -1, -1};
    const cudaError_t e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    std::printf("status %s\nexpired wait returned %d after %.1f ms\ncompleted wait returned %d\nafterwards %d %d\n",
                cudaGetErrorString(e), h[0], ms, h[1], h[2], h[3]);
    cudaFree(d);
    return (e == cudaSuccess && h[0] == 0 && h[1] == 1 && h[2] == 1 && h[3] == 1) ? 0 : 1;
}
