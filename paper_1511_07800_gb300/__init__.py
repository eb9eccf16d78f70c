"""GB300-native projection step of the simplified TPLS channel-flow solver."""
