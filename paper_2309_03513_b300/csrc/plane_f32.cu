// Plane-kernel instantiations for float (one translation unit per precision).
#include "plane_ops.cuh"

namespace tddft {

template <>
PlaneOps<float> plane_ops_for<float>(int n) {
  switch (n) {
    case 8:
      return PlaneLaunch<float, 8>::ops();
    case 12:
      return PlaneLaunch<float, 12>::ops();
    case 16:
      return PlaneLaunch<float, 16>::ops();
    case 24:
      return PlaneLaunch<float, 24>::ops();
    case 32:
      return PlaneLaunch<float, 32>::ops();
    case 36:
      return PlaneLaunch<float, 36>::ops();
    case 48:
      return PlaneLaunch<float, 48>::ops();
    case 64:
      return PlaneLaunch<float, 64>::ops();
    case 72:
      return PlaneLaunch<float, 72>::ops();
    case 80:
      return PlaneLaunch<float, 80>::ops();
    case 96:
      return PlaneLaunch<float, 96>::ops();
    case 108:
      return PlaneLaunch<float, 108>::ops();
    case 128:
      return PlaneLaunch<float, 128>::ops();
    default:
      return PlaneOps<float>{};
  }
}

}  // namespace tddft
