"""GB300-native sliced tensor-network contraction for random-circuit sampling."""
