// Pencil FFT passes instantiated for transform length 96.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(96)
}  // namespace lsgpu
