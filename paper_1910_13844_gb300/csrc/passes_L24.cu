// Pencil FFT passes instantiated for transform length 24.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(24)
}  // namespace lsgpu
