// cells.h -- the builder's Voronoi cells on the device.
#pragma once

#include "builder.h"
#include "kernels.h"

namespace p2m {

// The cell of every row of the KD tree in m (its points and child boxes on
// the device) as the host builder computes it (cell_core.h), one thread per
// cell.  Rows whose work overflows a buffer, whose cap loop cannot be
// chained or whose exact search gives up are marked in out.gave_up for the
// host.  Returns false on any CUDA error (nothing is kept; the host computes
// every cell).
bool cells_on_device(const DevView &m, const CellProblem &pb, CellResult &out);

}  // namespace p2m
