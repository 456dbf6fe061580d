// Ablation-variant kernels with value polynomials of degree 1 (all key sets).
#include "variants.cuh"

namespace efunc {
namespace variant {

EFUNC_VARIANT_DEGREE(1)

}  // namespace variant
}  // namespace efunc
