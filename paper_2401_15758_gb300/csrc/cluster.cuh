// Entry and exit of the thread-block-cluster sweep kernels.
#pragma once
#include <cooperative_groups.h>

namespace sc4 {

// Position in the cluster. In a cluster launch it also waits until every CTA of
// the cluster has started, so that no CTA reaches a peer's shared memory before
// the peer runs; cluster_leave closes a kernel so that no CTA exits while a peer
// may still read or write its shared memory.
template <bool CL>
__device__ __forceinline__ void cluster_pos(int& crank, int& csize) {
  if constexpr (CL) {
    auto c = cooperative_groups::this_cluster();
    crank = (int)c.block_rank();
    csize = (int)c.num_blocks();
    c.sync();
  } else {
    crank = 0;
    csize = 1;
  }
}

template <bool CL>
__device__ __forceinline__ void cluster_leave() {
  if constexpr (CL) cooperative_groups::this_cluster().sync();
}

}  // namespace sc4
