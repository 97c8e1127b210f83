// render_agg16.cu -- the aggregation forms of render_agg.cu for L = 16.
#define NGPRT_AGG_L16_UNIT
#include "render_agg.cu"
