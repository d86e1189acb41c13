// Pass kernels of the overlap losses (Sec. 5.C) for the input transform
// q = softmax(x); a translation unit of its own so that the build compiles the
// transforms in parallel.
#include "iou.cuh"

namespace augk {
template const IouPasses& iou_passes<XF_LOGITS>(int);
}  // namespace augk
