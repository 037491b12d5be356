"""GB300-native (sm_103a) online query path of GATE-style graph ANNS."""
