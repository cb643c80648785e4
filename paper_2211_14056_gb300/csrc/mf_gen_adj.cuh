// GENERATED by paper_2211_14056_gb300/gen_tables.py -- do not edit.
// Adjoint kernel, four gluons: where the adjoints of the four-gluon
// blocks are kept (the amplitude rows of one of the two colour orderings
// whose completions use the block; see full_block_slots).
#pragma once
#include <cstdint>
namespace mf {
// per completion path (walk order): slot | (block parity << 5) | (first use << 7)
static __constant__ uint8_t kG4Leaf4[24] = {151, 177, 149, 171, 143, 169, 150, 176, 147, 41, 173, 43, 148, 45, 178, 15, 48, 49, 50, 19, 20, 21, 22, 23};
// per four-gluon block (generator order): its slot
static __constant__ uint8_t kG4Slot4[12] = {23, 17, 21, 11, 15, 9, 22, 16, 19, 13, 20, 18};
}  // namespace mf
