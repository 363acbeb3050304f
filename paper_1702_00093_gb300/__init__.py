"""GB300-native EmbedJoin hot path: CGK embedding, bit-sampling LSH, sort-based
bucketing and banded bit-parallel verification, behind a C-ABI library."""
