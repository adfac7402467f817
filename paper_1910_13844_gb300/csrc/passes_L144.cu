// Pencil FFT passes instantiated for transform length 144 (72-point grids).
#include "passes.cuh"
namespace lsgpu {
LS_DEFINE_LENGTH(144)
}  // namespace lsgpu
