// ipm_school.cu -- the schoolbook family: c_k = sum_{i+j=k} a_i b_j by
// direct limb products, for products too small for the transform path to
// pay off (the definition of §1 computed as written; the paper compares
// against such plain algorithms in §4).
//
// One block per output coefficient (school.cuh, school_tile).
#include <cuda_runtime.h>

#include "ipm_internal.h"
#include "school.cuh"

namespace ipm {
namespace {

constexpr int SCHOOL_THREADS = 128;

__global__ void __launch_bounds__(SCHOOL_THREADS) k_school(const __grid_constant__ KParams P, const uint32_t *__restrict__ a,
                                                           const uint8_t *__restrict__ an,
                                                           const uint32_t *__restrict__ b,
                                                           const uint8_t *__restrict__ bn, uint32_t *__restrict__ c,
                                                           uint8_t *__restrict__ cn) {
    extern __shared__ __align__(16) unsigned char smem[];
    // several products of one shape (Karatsuba leaves): product blockIdx.y,
    // operands and result back to back
    const int64_t y = blockIdx.y;
    school_tile(P, blockIdx.x, a + y * P.na * P.la, an + y * P.na, b + y * P.nb * P.lb, bn + y * P.nb,
                c + y * P.nc * P.lc, cn + y * P.nc, smem);
}

}  // namespace

size_t school_smem(const KParams &kp) { return ((size_t)kp.la + kp.lb + 1) * (sizeof(long long) + sizeof(uint32_t)); }

int launch_school_batch(const KParams &kp, const uint32_t *a, const uint8_t *an, const uint32_t *b,
                        const uint8_t *bn, uint32_t *c, uint8_t *cn, int64_t count, void *stream) {
    dim3 grid((unsigned)kp.nc, (unsigned)count, 1);
    k_school<<<grid, SCHOOL_THREADS, school_smem(kp), (cudaStream_t)stream>>>(kp, a, an, b, bn, c, cn);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_school(const ShapePlan &sp, const uint32_t *a, const uint8_t *an, const uint32_t *b, const uint8_t *bn,
                  uint32_t *c, uint8_t *cn, void *stream) {
    const KParams &kp = sp.kp;
    k_school<<<(unsigned)kp.nc, SCHOOL_THREADS, school_smem(kp), (cudaStream_t)stream>>>(kp, a, an, b, bn, c, cn);
    note_launches(1);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace ipm
