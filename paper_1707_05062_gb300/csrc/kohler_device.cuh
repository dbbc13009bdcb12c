// Device code of libkohler, one header per pass; kohler_common.cuh states the
// method and the exact rewrite that every pass feeds.
#pragma once
#include "kohler_common.cuh"
#include "kohler_u16.cuh"
#include "kohler_u8r.cuh"
#include "kohler_u8h.cuh"
#include "kohler_u8n.cuh"
#include "kohler_pairs.cuh"
#include "kohler_thresholds.cuh"
