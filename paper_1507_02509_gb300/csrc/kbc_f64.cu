// Kernel instantiations for the CodecF64 storage codec (see kbc_lattice.cuh).
#define KBC_CODEC_TU 1
#include "kbc_launch.cuh"

namespace kbc {
KBC_DEFINE_CODEC(CodecF64)
}  // namespace kbc
