// Pencil FFT passes instantiated for transform length 192.
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(192)
}  // namespace lsgpu
