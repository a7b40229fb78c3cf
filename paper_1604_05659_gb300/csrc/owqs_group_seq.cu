// One slice of the complex64 pass-group kernels compiled for fixed
// register-slot sequences: this translation unit is compiled once per slice
// (-DOWQS_SEQ_SLICE=0 .. kGroupSeqSlices-1) and instantiates the sequences
// i of owqs_group_sequences.inc with i % kGroupSeqSlices == OWQS_SEQ_SLICE.
#include "owqs_group_c64.cuh"

#ifndef OWQS_SEQ_SLICE
#define OWQS_SEQ_SLICE 0
#endif

namespace owqs {

static_assert(OWQS_SEQ_SLICE >= 0 && OWQS_SEQ_SLICE < kGroupSeqSlices, "slice index");

template <int I>
static cudaError_t launch_group_sequence(const GroupParams& G, uint32_t code, cudaStream_t s, bool* launched) {
  if constexpr (I < kNumGroupSequences) {
    constexpr uint32_t C = kGroupSequences[I];
    constexpr int MM = (int)((C >> 28) & 7u);
    static_assert(MM >= 1 && MM <= kGroupRegMax && ((C >> 24) & 15u) >= 2 && ((C >> 24) & 15u) <= kGroupMax,
                  "sequence code");
    if (code == C) {
      *launched = true;
      // the kernel's sequence: the slots, k and the exact-half bit (M is its own parameter)
      return launch_group_t<MM, group_tile_bits(OWQS_C64, MM)>(k_group<MM, false, (C & 0x8fffffffu)>, G, s);
    }
    return launch_group_sequence<I + kGroupSeqSlices>(G, code, s, launched);
  } else {
    return cudaSuccess;
  }
}

template <>
cudaError_t launch_group_seq_slice<OWQS_SEQ_SLICE>(const GroupParams& G, uint32_t code, cudaStream_t s,
                                                   bool* launched) {
  return launch_group_sequence<OWQS_SEQ_SLICE>(G, code, s, launched);
}

}  // namespace owqs
