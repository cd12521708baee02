"""GB300-native periodic treecode force path (see ``nbody`` for the binding)."""
