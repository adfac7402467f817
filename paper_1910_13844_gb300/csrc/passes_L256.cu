// Pencil FFT passes instantiated for transform length 256.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(256)
}  // namespace lsgpu
