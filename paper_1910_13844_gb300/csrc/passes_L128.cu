// Pencil FFT passes instantiated for transform length 128.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(128)
}  // namespace lsgpu
