// Pencil FFT passes instantiated for transform length 64.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(64)
}  // namespace lsgpu
