/*
 * Device side of the synthetic generator: fills a device buffer with the
 * same bytes synth_generate_cpu writes, so full-size workloads need no host
 * generation or upload.  Runs the integer-only sampler of synth.h.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "synth.h"

__global__ void synth_kernel(uint8_t *__restrict__ out, int64_t n_frames,
                             int64_t frame0, int32_t M, int32_t N,
                             int32_t layout, uint32_t k0, uint32_t k1,
                             const uint32_t *__restrict__ thr_clean,
                             const syn_frame_t *__restrict__ frames,
                             const uint32_t *__restrict__ thr_rfi)
{
    const int32_t npair = (N + 1) / 2;
    const int64_t per_frame = (int64_t)M * npair;
    const int64_t total = n_frames * per_frame;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
         idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t f = idx / per_frame;
        int64_t rem = idx - f * per_frame;
        int32_t t = (int32_t)(rem / npair);
        int32_t ip = (int32_t)(rem - (int64_t)t * npair);
        syn_frame_t fr = frames[f];
        uint8_t b[2];
        syn_pair(k0, k1, (uint32_t)(frame0 + f), (uint32_t)t, (uint32_t)ip, N,
                 thr_clean, &fr, thr_rfi, b);
        uint8_t *fo = out + f * (int64_t)M * N;
        int32_t i = 2 * ip;
        if (layout == 0) {
            fo[(int64_t)t * N + i] = b[0];
            if (i + 1 < N)
                fo[(int64_t)t * N + i + 1] = b[1];
        } else {
            fo[(int64_t)i * M + t] = b[0];
            if (i + 1 < N)
                fo[(int64_t)(i + 1) * M + t] = b[1];
        }
    }
}

extern "C" int synth_generate_gpu(uint8_t *d_out, int64_t n_frames,
                                  int64_t frame0, int32_t M, int32_t N,
                                  int32_t layout, uint64_t seed,
                                  const uint32_t *d_thr_clean,
                                  const syn_frame_t *d_frames,
                                  const uint32_t *d_thr_rfi, void *stream)
{
    if (n_frames <= 0)
        return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
        cudaSuccess)
        return -1;
    int64_t total = n_frames * (int64_t)M * ((N + 1) / 2);
    int64_t blocks = (total + 255) / 256;
    int64_t cap = (int64_t)sms * 64;
    if (blocks > cap)
        blocks = cap;
    synth_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        d_out, n_frames, frame0, M, N, layout, (uint32_t)seed,
        (uint32_t)(seed >> 32), d_thr_clean, d_frames, d_thr_rfi);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
