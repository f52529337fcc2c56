// OVERLAP_PERSISTENT kernel instances with the tiles split along z (the zseg configuration field).
#define GIRIH_OVL_ZS true
#include "mwd_overlap_inst.cuh"
