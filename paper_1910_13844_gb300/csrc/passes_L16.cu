// Pencil FFT passes instantiated for transform length 16.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(16)
}  // namespace lsgpu
