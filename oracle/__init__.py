"""FP64 CPU oracle of the WeatherMesh-3 processor (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
import this package. The GPU library never depends on it.
"""
from .wm_oracle import (  # noqa: F401
    axis_window, block, block_fp8mlp, e4m3_decode, e4m3_round, fp8_mlp_scales, block_at_tokens, gelu, greedy_schedule, layer_norm, linear,
    neighbor_index, neighborhood_attention, processor, rel_l2, rollout, rope_angles, rope_pairs,
    rope_rotate, codec_patches_atm, codec_patches_sfc, codec_unpatch_atm, codec_unpatch_sfc, encode, decode,
)
