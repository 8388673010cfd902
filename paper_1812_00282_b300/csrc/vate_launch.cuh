// vate_launch.cuh -- host-side launch helper for kernels that touch an AT pool.
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include "vate_device.cuh"
#include "vate_internal.h"

namespace vate {

// Launch a kernel that reads or writes the AT pool.  When the handle asked for
// it, the launch carries an L2 access-policy window over the pool: hits are
// kept as persisting lines, so the pool (state kept from slice to slice)
// stays in L2 while the pairs and host lists stream through it.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pool(const Geom &G, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                               cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (G.l2_window_bytes) {
        attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[0].val.accessPolicyWindow.base_ptr = pool_mem(G);
        attr[0].val.accessPolicyWindow.num_bytes = G.l2_window_bytes;
        attr[0].val.accessPolicyWindow.hitRatio = G.l2_hit_ratio;
        attr[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        attr[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    count_launch();
    return e;
}

}  // namespace vate
