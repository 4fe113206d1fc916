// pack.h -- the builder's packing of the interception table on the device.
#pragma once

#include <cstdint>
#include <vector>

#include "builder.h"

namespace p2m {

// Pack the records (the parts' records with row >= 0, any order) into the
// table as the host builder does (pack_core.h): out's row_off, entries,
// chunk_off, chunks, super_off and supers, in the code frame qlo / qinv
// (quant.h).  bad_boxes counts entry codes outside their chunk's frame.
// Returns false when the device cannot do it (a row longer than its sort
// holds, a CUDA error): nothing is kept and the host packs.
bool pack_on_device(int64_t nv, const std::vector<PackPart> &parts, const float qlo[3],
                    const float qinv[3], Layout &out, int64_t &max_list, int64_t &bad_boxes);

}  // namespace p2m
