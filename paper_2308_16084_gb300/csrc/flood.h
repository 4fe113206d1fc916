// flood.h -- the flooding inspection (Alg. 1) of the builder on the device.
#pragma once

#include <cstdint>
#include <vector>

#include "builder.h"

namespace p2m {

// Flood every primitive of pb on the current device: one warp per
// primitive at a time (flood_warp.h) over the widened cells held in device
// memory.  out receives the records of the primitives finished on the
// device (in no particular order), gave_up[i] = 1 marks the primitives it
// gave up (a work polytope over its capacity, cap chaining or the visit
// limit: the host floods them), inspections the vertices inspected for the
// finished ones.  The records equal the host core's bit for bit: the same
// double-precision operations, compiled without fused multiply-adds.
// Returns false on any CUDA error (nothing is kept; the host floods all).
bool flood_on_device(const FloodProblem &pb, std::vector<FloodRec> &out,
                     std::vector<uint8_t> &gave_up, int64_t &inspections);

}  // namespace p2m
