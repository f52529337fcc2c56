// OVERLAP_PERSISTENT kernel instances on whole tiles.
#define GIRIH_OVL_ZS false
#include "mwd_overlap_inst.cuh"
