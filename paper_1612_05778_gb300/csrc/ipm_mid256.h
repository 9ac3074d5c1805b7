// ipm_mid256.h -- the middle pass in 256-thread blocks, two per SM, for
// single products and batched launches (ipm_kernels_mid256.cu).
#pragma once
#include <stddef.h>

#include "ipm_internal.h"

namespace ipm {

// Largest middle tile for which two 256-thread blocks share an SM.
constexpr size_t MID256_SMEM_MAX = 113 * 1024;

int set_kernel_attributes_mid256();
int launch_batch_middle256(const BatchLaunch &bl, void *stream);
int launch_middle256(const KParams &kp, size_t smem, void *stream);
bool mid256_ok(const KParams &kp, size_t smem_mid);

}  // namespace ipm
