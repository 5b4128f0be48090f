// Internal interface between the FGMRES driver (api.cu) and the learned
// coarse correction (api_net.cu).
#pragma once

#include "host.h"

namespace rp {

// z += gamma s / Nc * prolong(net(restrict(r1) Nc / s)), s = ||restrict(r1)||,
// on stream st; the transfer kernels return at once when kst->stop is set.
int net_correct(ras_pml_net* n, const c128* r1, c128* z, int nx, int ny, const KState* kst, cudaStream_t st);
// the coarse grid size of the network
int net_grid(const ras_pml_net* n);

}  // namespace rp
