// Pencil FFT passes instantiated for transform length 48.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(48)
}  // namespace lsgpu
