// The box-object model's physics and reset kernels with the box store: every
// node of the distance grid is recomputed from the scene's solid boxes (see
// gx_device.cuh) instead of read from the dense grid.  Same source as
// gx_boxes.cu.
#define GX_STATIC_STORE 1
#include "gx_boxes.cu"
