// Pencil FFT passes instantiated for transform length 32.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(32)
}  // namespace lsgpu
