// Pencil FFT passes instantiated for transform length 384.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(384)
}  // namespace lsgpu
